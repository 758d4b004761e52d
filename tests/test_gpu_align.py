"""Parity of sw_align (score, start/end point, CIGAR) with the CPU oracle.

Bit-exact: the CIGAR is the greedy traceback path (diagonal > I > D; open >
extend) from the end point, so a single differing op fails.  Small leaf and
checkpoint settings force many levels of the linear-space recursion, label
passes in both orientations and E/F source/sink states on small inputs.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from gen import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def sw():
    import paper_1304_5966_gb300 as m
    from paper_1304_5966_gb300 import build
    build.build()
    return m


@pytest.fixture(scope="module")
def ctx(sw):
    c = sw.sw_ctx_create(0, workspace_bytes=2 << 30)
    yield c
    c.close()


def _tuple(r):
    return (r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.cigar or "")


def _check(sw, ctx, a, b, sch=oracle.DNA, s=None, flags=0):
    want = oracle.align(a, b, sch)
    got = sw.sw_align(ctx, a, b, s, flags)
    assert _tuple(got) == _tuple(want), (len(a), len(b))
    return got


def _gappy_pair(n, seed):
    """A homologous pair with long insertions and deletions (E and F runs)."""
    a, b = synth.related_pair(n, seed=seed, sub_permille=80)
    st = synth.Rng(seed + 1000).stream()
    pieces, pos = [], 0
    while pos < len(b):
        step = st.int(50, 400)
        pieces.append(b[pos:pos + step])
        pos += step
        if st.int(0, 1):
            pos += st.int(5, 60)                                   # deletion in B
        else:
            pieces.append(synth.random_bases(st, st.int(5, 60)))   # insertion in B
    return a, np.concatenate(pieces).astype(np.uint8)


@pytest.mark.parametrize("n,m", [(1, 1), (5, 3), (64, 64), (255, 257), (300, 260), (700, 650),
                                 (1000, 999), (1500, 2600), (2600, 1500)])
def test_related_pairs(sw, ctx, n, m):
    a, b0 = synth.related_pair(max(n, m), seed=n * 31 + m)
    _check(sw, ctx, a[:n], b0[:m])


@pytest.mark.parametrize("seed", range(4))
def test_gappy_pairs(sw, ctx, seed):
    a, b = _gappy_pair(2500, seed)
    _check(sw, ctx, a, b)
    _check(sw, ctx, b, a)


@pytest.mark.parametrize("leaf,ck", [(256, 1), (1024, 1), (4096, 2), (256, 3)])
def test_deep_recursion(sw, ctx, leaf, ck):
    ctx.set_option(sw.SW_OPT_LEAF_CELLS, leaf)
    ctx.set_option(sw.SW_OPT_CKPT_BANDS, ck)
    try:
        for seed in range(3):
            a, b = _gappy_pair(1800 + 300 * seed, 40 + seed)
            got = _check(sw, ctx, a, b)
            assert got.stats["levels"] >= 2
            _check(sw, ctx, b[:900], a[:1700])
    finally:
        ctx.set_option(sw.SW_OPT_LEAF_CELLS, 1 << 16)
        ctx.set_option(sw.SW_OPT_CKPT_BANDS, 0)


def test_schemes(sw, ctx):
    a, b = _gappy_pair(1200, 7)
    for sch in [oracle.Scheme(2, -1, 2, 1), oracle.Scheme(1, -1, 1, 1), oracle.Scheme(3, -2, 4, 4),
                oracle.Scheme(5, -4, 10, 1)]:
        s = sw.Scheme(sch.match, sch.mismatch, sch.gap_open, sch.gap_extend)
        _check(sw, ctx, a, b, sch, s)
    ctx.set_option(sw.SW_OPT_LEAF_CELLS, 256)
    ctx.set_option(sw.SW_OPT_CKPT_BANDS, 1)
    try:
        for sch in [oracle.Scheme(2, -1, 2, 1), oracle.Scheme(1, -1, 1, 1)]:
            s = sw.Scheme(sch.match, sch.mismatch, sch.gap_open, sch.gap_extend)
            _check(sw, ctx, a, b, sch, s)
    finally:
        ctx.set_option(sw.SW_OPT_LEAF_CELLS, 1 << 16)
        ctx.set_option(sw.SW_OPT_CKPT_BANDS, 0)


def test_tie_heavy(sw, ctx):
    cases = [
        (np.tile(np.array([0, 1], np.uint8), 700), np.tile(np.array([0, 1], np.uint8), 650)),
        (np.tile(np.array([0, 0, 1], np.uint8), 400), np.tile(np.array([0, 1], np.uint8), 500)),
        (np.zeros(900, np.uint8), np.zeros(1300, np.uint8)),
    ]
    ctx.set_option(sw.SW_OPT_LEAF_CELLS, 1024)
    ctx.set_option(sw.SW_OPT_CKPT_BANDS, 1)
    try:
        for a, b in cases:
            _check(sw, ctx, a, b)
            _check(sw, ctx, b, a)
    finally:
        ctx.set_option(sw.SW_OPT_LEAF_CELLS, 1 << 16)
        ctx.set_option(sw.SW_OPT_CKPT_BANDS, 0)


def test_prune_off_identical(sw, ctx):
    a, b = _gappy_pair(3000, 11)
    r1 = sw.sw_align(ctx, a, b)
    r2 = sw.sw_align(ctx, a, b, flags=sw.SW_FLAG_NO_PRUNE)
    assert _tuple(r1) == _tuple(r2)


def test_alphabet5_and_device_input(sw, ctx):
    import torch
    st = synth.Rng(21).stream()
    a = st.below(1500, 5).astype(np.uint8)
    b = a.copy()
    b[::9] = 4
    b = np.concatenate([b[:700], b[760:]]).astype(np.uint8)
    sch = oracle.Scheme(1, -3, 5, 2, alphabet=5)
    _check(sw, ctx, a, b, sch, sw.Scheme(1, -3, 5, 2, alphabet=5))
    a2, b2 = _gappy_pair(2000, 5)
    want = oracle.align(a2, b2)
    got = sw.sw_align(ctx, torch.from_numpy(a2).cuda(), torch.from_numpy(b2).cuda())
    assert _tuple(got) == _tuple(want)


def test_zero_score_and_empty(sw, ctx):
    mat = tuple(1 if x == y else -1 for x in range(4) for y in range(4))
    st = synth.Rng(8).stream()
    a = st.below(300, 2).astype(np.uint8)
    b = (st.below(400, 2) + 2).astype(np.uint8)
    r = sw.sw_align(ctx, a, b, sw.Scheme(alphabet=4, matrix=mat))
    assert _tuple(r) == (0, -1, -1, -1, -1, "")
    r = sw.sw_align(ctx, a[:0], b)
    assert _tuple(r) == (0, -1, -1, -1, -1, "")


def test_pair_1k_golden(sw, ctx):
    g = json.load(open(os.path.join(HERE, "golden", "pair_1k.json")))
    a, b = synth.pair_1k()
    r = sw.sw_align(ctx, a, b)
    assert _tuple(r) == (g["score"], g["a_begin"], g["a_end"], g["b_begin"], g["b_end"], g["cigar"])


def test_pair_100k_golden(sw, ctx):
    g = json.load(open(os.path.join(HERE, "golden", "pair_100k.json")))
    a, b = synth.pair_100k()
    r = sw.sw_align(ctx, a, b)
    assert (r.score, r.a_begin, r.a_end, r.b_begin, r.b_end) == \
        (g["score"], g["a_begin"], g["a_end"], g["b_begin"], g["b_end"])
    assert len(r.cigar) == g["cigar_len"]
    assert hashlib.sha256(r.cigar.encode()).hexdigest() == g["cigar_sha256"]


def test_start_pass_lanes_identical(sw, ctx):
    """The start-point pass on int16x2 offset lanes equals the int32 pass."""
    a, b = _gappy_pair(6000, 71)
    r16 = sw.sw_align(ctx, a, b)
    ctx.set_option(sw.SW_OPT_FORWARD_LANES, 32)
    try:
        r32 = sw.sw_align(ctx, a, b)
    finally:
        ctx.set_option(sw.SW_OPT_FORWARD_LANES, 0)
    assert _tuple(r16) == _tuple(r32) == _tuple(oracle.align(a, b))


@pytest.mark.parametrize("rpt", [4, 8, 16])
def test_offset_lanes_band_heights(sw, ctx, rpt):
    """int16x2 offset lanes at every band height, pruning on and off: pruned
    bands whose state is all sentinels must re-centre on the next finite input."""
    ctx.set_option(sw.SW_OPT_FORWARD_LANES, 16)
    ctx.set_option(sw.SW_OPT_ROWS_PER_THREAD, rpt)
    try:
        for seed, (n, m) in enumerate([(700, 650), (2600, 1500), (1000, 999), (4100, 3900)]):
            a, b0 = synth.related_pair(max(n, m), seed=n * 31 + m)
            a, b = a[:n], b0[:m]
            want = _tuple(oracle.align(a, b))
            assert _tuple(sw.sw_align(ctx, a, b)) == want
            assert _tuple(sw.sw_align(ctx, a, b, flags=sw.SW_FLAG_NO_PRUNE)) == want
        a, b = _gappy_pair(5000, 81)
        assert _tuple(sw.sw_align(ctx, a, b)) == _tuple(oracle.align(a, b))
    finally:
        ctx.set_option(sw.SW_OPT_FORWARD_LANES, 0)
        ctx.set_option(sw.SW_OPT_ROWS_PER_THREAD, 0)


def test_local_pass_one_cta_per_sm(sw, ctx):
    """A local pass with bands enough for the one-CTA-per-SM layout (each
    scheduler on consecutive bands, 256-row bands): score and end equal the
    oracle's, pruning on and off, and the layout was the one used."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 2 * sms * 20 * 256 + 70_001           # past the layout's threshold, ragged last band
    st = synth.Rng(97).stream()
    a = synth.random_bases(st, n)
    core = a[n - 300_000:n - 299_400].copy()
    b = np.concatenate([synth.random_bases(st, 50), synth.mutate(st, core), synth.random_bases(st, 40)])
    want = oracle.local_score(a, b)           # (score, a_end, b_end); the planted copy scores far above 0
    ctx.set_option(sw.SW_OPT_FORWARD_LANES, 16)
    ctx.set_option(sw.SW_OPT_ROWS_PER_THREAD, 4)
    try:
        for fl in (0, sw.SW_FLAG_NO_PRUNE):
            r = sw.sw_score(ctx, a, b, flags=fl)
            assert r.stats["cta_warps"] == 20
            assert (r.score, r.a_end, r.b_end) == want
    finally:
        ctx.set_option(sw.SW_OPT_FORWARD_LANES, 0)
        ctx.set_option(sw.SW_OPT_ROWS_PER_THREAD, 0)


def test_pair_5m_full_size():
    """The 5,000,000 x 4,948,987 pair in the benchmark's launch configuration
    (24 GiB workspace, default options).  The oracle cannot run the whole
    matrix, so the checks are the ones that hold at any size plus sampled
    sub-problems it solves one by one:
      * pruning on and off give the same score and end point;
      * the CIGAR rescored on the CPU equals the score and consumes exactly
        [a_begin, a_end) x [b_begin, b_end), beginning and ending with a match;
      * windows of the path between two nodes in state H are exactly the
        oracle's greedy traceback of that sub-problem (the sub-path property
        that test_oracle pins on exhaustive cases)."""
    import paper_1304_5966_gb300 as sw
    import torch
    a, b = synth.pair_5m()
    c = sw.sw_ctx_create(0, workspace_bytes=24 << 30)
    try:
        ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
        r = sw.sw_align(c, ta, tb)
        rn = sw.sw_score(c, ta, tb, flags=sw.SW_FLAG_NO_PRUNE)
    finally:
        c.close()
    assert r.score > 1_000_000
    assert (rn.score, rn.a_end, rn.b_end) == (r.score, r.a_end, r.b_end)
    ops = oracle.cigar_to_ops(r.cigar)
    asub, bsub = a[r.a_begin:r.a_end], b[r.b_begin:r.b_end]
    assert oracle.rescore(asub, bsub, ops) == (r.score, len(asub), len(bsub))
    assert r.cigar.endswith("=") and r.cigar[:r.cigar.index("=")].isdigit()
    # positions (i, j) before each op; a node after an 'M' op is in state H
    steps = np.frombuffer(ops.encode(), dtype=np.uint8)
    di = np.concatenate([[0], np.cumsum((steps == ord("M")) | (steps == ord("I")))])
    dj = np.concatenate([[0], np.cumsum((steps == ord("M")) | (steps == ord("D")))])
    h_nodes = np.flatnonzero(steps == ord("M")) + 1           # op index just after an 'M'
    st = synth.Rng(5005).stream()
    for _ in range(24):
        k0 = int(h_nodes[st.int(0, len(h_nodes) - 1)])
        k1 = int(h_nodes[np.searchsorted(h_nodes, min(k0 + st.int(500, 4000), int(h_nodes[-1])))])
        if k1 <= k0:
            continue
        i0, j0, i1, j1 = int(di[k0]), int(dj[k0]), int(di[k1]), int(dj[k1])
        assert oracle.verify_path(asub[i0:i1], bsub[j0:j1], ops[k0:k1]) == 0, (k0, k1)
