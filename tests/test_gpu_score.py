"""Parity of the CUDA forward pass (sw_score) with the CPU oracle, through the C ABI.

Bit-exact: score and end point (first cell with H = S in row-major order).
"""
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
    c = sw.sw_ctx_create(0, workspace_bytes=1 << 30)
    yield c
    c.close()


def _want(a, b, sch=oracle.DNA):
    return oracle.local_score(a, b, sch)


def _got(sw, ctx, a, b, sch=None, flags=0):
    r = sw.sw_score(ctx, a, b, sch, flags)
    return r.score, (r.a_end if r.score else -1), (r.b_end if r.score else -1)


SHAPES = [(1, 1), (1, 40), (40, 1), (31, 33), (32, 32), (33, 31), (255, 257), (511, 513),
          (512, 512), (513, 700), (1000, 999), (1537, 1100), (2049, 3000), (4100, 2500)]


@pytest.mark.parametrize("n,m", SHAPES)
def test_random_related_pairs(sw, ctx, n, m):
    a, b0 = synth.related_pair(max(n, m), seed=n * 7919 + m)
    a, b = a[:n], b0[:m]
    assert _got(sw, ctx, a, b) == _want(a, b)


@pytest.mark.parametrize("seed", range(6))
def test_unrelated_pairs(sw, ctx, seed):
    a, b = synth.random_pair(700 + 97 * seed, 1500 - 61 * seed, seed=seed)
    assert _got(sw, ctx, a, b) == _want(a, b)


@pytest.mark.parametrize("rpt", [8, 16, 24, 32])
def test_rows_per_thread_variants(sw, ctx, rpt):
    ctx.set_option(sw.SW_OPT_ROWS_PER_THREAD, rpt)
    try:
        for seed in range(3):
            a, b = synth.related_pair(3000 + 13 * seed, seed=100 + seed)
            assert _got(sw, ctx, a, b) == _want(a, b)
            assert _got(sw, ctx, a, b, flags=sw.SW_FLAG_NO_PRUNE) == _want(a, b)
    finally:
        ctx.set_option(sw.SW_OPT_ROWS_PER_THREAD, 0)


def test_tie_heavy_inputs(sw, ctx):
    cases = [
        (np.zeros(700, np.uint8), np.zeros(900, np.uint8)),                       # homopolymers
        (np.tile(np.array([0, 1], np.uint8), 600), np.tile(np.array([0, 1], np.uint8), 450)),
        (np.tile(np.array([0, 1, 2], np.uint8), 400), np.tile(np.array([2, 0, 1], np.uint8), 500)),
        (np.tile(np.array([0, 0, 1], np.uint8), 333), np.tile(np.array([0, 1], np.uint8), 777)),
    ]
    for a, b in cases:
        assert _got(sw, ctx, a, b) == _want(a, b)
        assert _got(sw, ctx, b, a) == _want(b, a)


def test_schemes_and_alphabets(sw, ctx):
    a, b = synth.related_pair(1500, seed=5, sub_permille=200)
    for sch in [oracle.Scheme(2, -1, 2, 1), oracle.Scheme(1, -1, 1, 1), oracle.Scheme(5, -4, 10, 1),
                oracle.Scheme(3, -2, 4, 4)]:
        s = sw.Scheme(sch.match, sch.mismatch, sch.gap_open, sch.gap_extend)
        assert _got(sw, ctx, a, b, s) == _want(a, b, sch)
    # 5-letter alphabet with N (two profile words)
    st = synth.Rng(9).stream()
    a5 = st.below(2000, 5).astype(np.uint8)
    b5 = a5.copy()
    b5[::7] = 4
    sch5 = oracle.Scheme(1, -3, 5, 2, alphabet=5)
    assert _got(sw, ctx, a5, b5, sw.Scheme(1, -3, 5, 2, alphabet=5)) == _want(a5, b5, sch5)
    # explicit 8-letter matrix
    mat = tuple(int(v) for v in (np.arange(64).reshape(8, 8) % 7 - 4).ravel())
    a8 = st.below(1200, 8).astype(np.uint8)
    b8 = st.below(1300, 8).astype(np.uint8)
    assert _got(sw, ctx, a8, b8, sw.Scheme(alphabet=8, matrix=mat)) == \
        _want(a8, b8, oracle.Scheme(alphabet=8, matrix=mat))


def test_empty_and_degenerate(sw, ctx):
    assert _got(sw, ctx, np.zeros(0, np.uint8), np.zeros(5, np.uint8)) == (0, -1, -1)
    assert _got(sw, ctx, np.zeros(5, np.uint8), np.zeros(0, np.uint8)) == (0, -1, -1)
    # nothing aligns with a positive score: codes {0,1} against {2,3}
    mat = tuple(1 if x == y else -1 for x in range(4) for y in range(4))
    st = synth.Rng(8).stream()
    a = st.below(300, 2).astype(np.uint8)
    b = (st.below(400, 2) + 2).astype(np.uint8)
    assert _got(sw, ctx, a, b, sw.Scheme(alphabet=4, matrix=mat)) == (0, -1, -1)
    # a scheme with no positive score cannot define a local alignment: rejected
    with pytest.raises(sw.SwError) as e:
        sw.sw_score(ctx, a, b, sw.Scheme(alphabet=4, matrix=tuple([-1] * 16)))
    assert e.value.status == sw.SW_EINVAL


def test_invalid_inputs(sw, ctx):
    with pytest.raises(sw.SwError) as e:
        sw.sw_score(ctx, np.array([0, 1, 9], np.uint8), np.array([0, 1], np.uint8))
    assert e.value.status == sw.SW_EINVAL
    with pytest.raises(sw.SwError) as e:
        sw.sw_score(ctx, np.array([0, 1], np.uint8), np.array([0, 1], np.uint8), sw.Scheme(1, -3, 1, 2))
    assert e.value.status == sw.SW_EINVAL


def test_device_inputs(sw, ctx):
    import torch
    a, b = synth.related_pair(5000, seed=42)
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b).cuda()
    assert _got(sw, ctx, ta, tb) == _want(a, b)


def test_pair_1k_golden(sw, ctx):
    g = json.load(open(os.path.join(HERE, "golden", "pair_1k.json")))
    a, b = synth.pair_1k()
    assert _got(sw, ctx, a, b) == (g["score"], g["a_end"], g["b_end"])


def test_pair_100k_golden(sw, ctx):
    g = json.load(open(os.path.join(HERE, "golden", "pair_100k.json")))
    a, b = synth.pair_100k()
    assert _got(sw, ctx, a, b) == (g["score"], g["a_end"], g["b_end"])
    assert _got(sw, ctx, a, b, flags=sw.SW_FLAG_NO_PRUNE) == (g["score"], g["a_end"], g["b_end"])


def test_plain_path_matches(sw, ctx):
    for n, m in [(1, 1), (100, 37), (1000, 1200), (3000, 2900)]:
        a, b0 = synth.related_pair(max(n, m), seed=n + m)
        a, b = a[:n], b0[:m]
        r = sw.sw_score_plain(ctx, a, b)
        assert (r.score, r.a_end if r.score else -1, r.b_end if r.score else -1) == _want(a, b)


def test_bounded_wait_timeout_is_reported(sw, ctx):
    """A band that never publishes makes the next band's bounded wait expire;
    the kernel stops itself and the call returns SW_ETIMEOUT (no fault, no hang)."""
    a, b = synth.related_pair(20000, seed=3)
    ctx.set_option(sw.SW_OPT_TIMEOUT_MS, 300)
    ctx.set_option(sw.SW_OPT_FAULT_BAND, 2)
    try:
        with pytest.raises(sw.SwError) as e:
            sw.sw_score(ctx, a, b)
        assert e.value.status == sw.SW_ETIMEOUT
    finally:
        ctx.set_option(sw.SW_OPT_FAULT_BAND, -1)
        ctx.set_option(sw.SW_OPT_TIMEOUT_MS, 2000)
    # the context stays usable
    assert _got(sw, ctx, a[:3000], b[:3000]) == _want(a[:3000], b[:3000])


@pytest.mark.parametrize("lanes", [16, 32])
def test_forward_lanes_identical(sw, ctx, lanes):
    """int16x2 lanes with per-warp offsets and int32 lanes give the same result,
    including on scores far beyond int16 (the 100 kbp pair scores 41,971)."""
    ctx.set_option(sw.SW_OPT_FORWARD_LANES, lanes)
    try:
        a, b = synth.pair_100k()
        g = json.load(open(os.path.join(HERE, "golden", "pair_100k.json")))
        assert _got(sw, ctx, a, b) == (g["score"], g["a_end"], g["b_end"])
        assert _got(sw, ctx, a, b, flags=sw.SW_FLAG_NO_PRUNE) == (g["score"], g["a_end"], g["b_end"])
        for seed in range(4):
            x, y = synth.related_pair(4000 + 777 * seed, seed=300 + seed)
            assert _got(sw, ctx, x, y) == _want(x, y)
            assert _got(sw, ctx, y[:2500], x) == _want(y[:2500], x)
        # a scheme whose value spread does not fit int16 falls back to int32 lanes
        s = sw.Scheme(40, -30, 60, 20)
        x, y = synth.related_pair(3000, seed=400)
        assert _got(sw, ctx, x, y, s) == _want(x, y, oracle.Scheme(40, -30, 60, 20))
    finally:
        ctx.set_option(sw.SW_OPT_FORWARD_LANES, 0)
