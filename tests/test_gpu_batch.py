"""Parity of the batched path (sw_align_batch) with the CPU oracle.

Pairs of very different lengths share one persistent launch; pairs are
transposed when B is longer, run on int16x2 lanes when their score bound fits,
and re-run on int32 lanes after an int16 overflow.  Every pair must match the
oracle bit for bit (score, end point; start point and CIGAR when aligned), and
the batch must match the single-pair entry points.
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
    c = sw.sw_ctx_create(0, workspace_bytes=4 << 30)
    yield c
    c.close()


def _mixed_pairs(count, seed, lo=1, hi=3000):
    st = synth.Rng(seed).stream()
    pairs = []
    for t in range(count):
        n = int(synth.log_uniform_int(st, lo, hi, 1)[0])
        m = int(synth.log_uniform_int(st, lo, hi, 1)[0])
        if t % 3 == 0:
            a, b = synth.random_pair(n, m, seed=seed * 1000 + t)
        else:
            a, b0 = synth.related_pair(max(n, m), seed=seed * 1000 + t)
            a, b = a[:n], b0[:m]
        pairs.append((a, b))
    pairs.append((np.zeros(0, np.uint8), np.zeros(7, np.uint8)))     # empty side
    pairs.append((np.array([2], np.uint8), np.array([2], np.uint8)))  # 1 x 1
    return pairs


def _se(r):
    return (r.score, r.a_end, r.b_end) if r.score else (0, -1, -1)


def test_score_only_mixed(sw, ctx):
    pairs = _mixed_pairs(150, 1)
    got = sw.sw_align_batch(ctx, pairs, flags=sw.SW_FLAG_SCORE_ONLY)
    for (a, b), r in zip(pairs, got):
        S, ei, ej = oracle.local_score(a, b)
        assert _se(r) == ((S, ei, ej) if S else (0, -1, -1)), (len(a), len(b))


@pytest.mark.parametrize("flags", ["FORCE_INT32", "NO_PRUNE"])
def test_score_only_variants_identical(sw, ctx, flags):
    pairs = _mixed_pairs(80, 2)
    base = sw.sw_align_batch(ctx, pairs, flags=sw.SW_FLAG_SCORE_ONLY)
    other = sw.sw_align_batch(ctx, pairs, flags=sw.SW_FLAG_SCORE_ONLY | getattr(sw, "SW_FLAG_" + flags))
    assert [_se(r) for r in base] == [_se(r) for r in other]


def test_int16_overflow_rerun(sw, ctx):
    # match 100: bound 100 * min(n, m) exceeds int16 for the longer pairs; forcing
    # int16 lanes must detect it and re-run those pairs on int32 lanes
    sch = oracle.Scheme(100, -90, 120, 40)
    s = sw.Scheme(100, -90, 120, 40)
    pairs = _mixed_pairs(40, 3, lo=100, hi=1500)
    got = sw.sw_align_batch(ctx, pairs, s, flags=sw.SW_FLAG_SCORE_ONLY | sw.SW_FLAG_FORCE_INT16)
    assert got[0].stats["int16_reruns"] > 0
    for (a, b), r in zip(pairs, got):
        S, ei, ej = oracle.local_score(a, b, sch)
        assert _se(r) == ((S, ei, ej) if S else (0, -1, -1))


def test_align_mixed(sw, ctx):
    pairs = _mixed_pairs(40, 4, lo=1, hi=1500)
    got = sw.sw_align_batch(ctx, pairs)
    for (a, b), r in zip(pairs, got):
        w = oracle.align(a, b)
        assert (r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.cigar or "") == \
            (w.score, w.a_begin, w.a_end, w.b_begin, w.b_end, w.cigar), (len(a), len(b))


def test_batch_equals_single(sw, ctx):
    pairs = _mixed_pairs(12, 5, lo=200, hi=2500)
    got = sw.sw_align_batch(ctx, pairs)
    for (a, b), r in zip(pairs, got):
        one = sw.sw_align(ctx, a, b)
        assert (r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.cigar) == \
            (one.score, one.a_begin, one.a_end, one.b_begin, one.b_end, one.cigar)


def test_asymmetric_matrix(sw, ctx):
    # s(x, y) != s(y, x): transposed problems must use the transposed table
    mat = (2, -1, -3, 0,
           -2, 3, -1, -4,
           0, -3, 1, -2,
           -1, -2, -4, 2)
    sch = oracle.Scheme(alphabet=4, matrix=mat)
    s = sw.Scheme(alphabet=4, matrix=mat)
    pairs = _mixed_pairs(30, 6, lo=50, hi=1200)
    got = sw.sw_align_batch(ctx, pairs, s, flags=sw.SW_FLAG_SCORE_ONLY)
    for (a, b), r in zip(pairs, got):
        S, ei, ej = oracle.local_score(a, b, sch)
        assert _se(r) == ((S, ei, ej) if S else (0, -1, -1))
    for (a, b) in pairs[:8]:
        w = oracle.align(a, b, sch)
        r = sw.sw_align(ctx, a, b, s)
        assert (r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.cigar or "") == \
            (w.score, w.a_begin, w.a_end, w.b_begin, w.b_end, w.cigar)
    # a wide pair (B much longer) forces transposed label passes
    a, b = synth.related_pair(2500, seed=61)
    a = a[700:1500]
    w = oracle.align(a, b, sch)
    ctx.set_option(sw.SW_OPT_CKPT_BANDS, 1)
    ctx.set_option(sw.SW_OPT_LEAF_CELLS, 256)
    try:
        r = sw.sw_align(ctx, a, b, s)
    finally:
        ctx.set_option(sw.SW_OPT_CKPT_BANDS, 0)
        ctx.set_option(sw.SW_OPT_LEAF_CELLS, 1 << 16)
    assert (r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.cigar or "") == \
        (w.score, w.a_begin, w.a_end, w.b_begin, w.b_end, w.cigar)


def test_device_inputs(sw, ctx):
    import torch
    pairs = _mixed_pairs(20, 7, lo=10, hi=2000)
    dev = [(torch.from_numpy(a.copy()).cuda(), torch.from_numpy(b.copy()).cuda()) for a, b in pairs]
    got = sw.sw_align_batch(ctx, dev)
    for (a, b), r in zip(pairs, got):
        w = oracle.align(a, b)
        assert (r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.cigar or "") == \
            (w.score, w.a_begin, w.a_end, w.b_begin, w.b_end, w.cigar)


def test_batch_4096_golden(sw, ctx):
    g = json.load(open(os.path.join(HERE, "golden", "batch_4096.json")))
    pairs = synth.batch_pairs()
    got = sw.sw_align_batch(ctx, pairs, flags=sw.SW_FLAG_SCORE_ONLY)
    want = [tuple(x) if x[0] else (0, -1, -1) for x in g["score_end"]]
    assert [_se(r) for r in got] == want


def _strand_pairs(seed):
    """Pairs whose best strand is B as given, its reverse complement, or
    either (a B that is its own reverse complement: a tie)."""
    st = synth.Rng(seed).stream()
    pairs = []
    for t in range(36):
        n = int(synth.log_uniform_int(st, 20, 2500, 1)[0])
        a, b = synth.related_pair(n, seed=seed * 100 + t)
        if t % 3 == 1:
            b = synth.revcomp(b)
        elif t % 3 == 2:
            a, b = synth.random_pair(n, int(synth.log_uniform_int(st, 1, 2500, 1)[0]), seed=seed * 100 + t)
        pairs.append((a, b))
    x = synth.random_bases(st, 300)
    pairs.append((synth.random_bases(st, 900), np.concatenate([x, synth.revcomp(x)])))   # tie
    pairs.append((x.copy(), np.concatenate([x, synth.revcomp(x)])))                      # tie, high score
    pairs.append((x.copy(), np.zeros(0, np.uint8)))                                      # empty B
    return pairs


def _best_strand(a, b, score_only):
    """The oracle on both strands; the reverse one only when strictly better."""
    rb = synth.revcomp(b)
    if score_only:
        f, r = oracle.local_score(a, b), oracle.local_score(a, rb)
        w, strand = (r, 1) if r[0] > f[0] else (f, 0)
        return (w if w[0] else (0, -1, -1)), strand
    f, r = oracle.align(a, b), oracle.align(a, rb)
    w, strand = (r, 1) if r.score > f.score else (f, 0)
    return (w.score, w.a_begin, w.a_end, w.b_begin, w.b_end, w.cigar), strand


def test_both_strands(sw, ctx):
    """SW_FLAG_BOTH_STRANDS: each pair runs against B and revcomp(B) in one batch
    and keeps the strand with the higher score (forward on a tie), score-only and
    aligned, host and device inputs."""
    import torch
    pairs = _strand_pairs(5)
    so = sw.sw_align_batch(ctx, pairs, flags=sw.SW_FLAG_SCORE_ONLY | sw.SW_FLAG_BOTH_STRANDS)
    al = sw.sw_align_batch(ctx, pairs, flags=sw.SW_FLAG_BOTH_STRANDS)
    dev = [(torch.from_numpy(a.copy()).cuda(), torch.from_numpy(b.copy()).cuda()) for a, b in pairs]
    ad = sw.sw_align_batch(ctx, dev, flags=sw.SW_FLAG_BOTH_STRANDS)
    strands = []
    for k, (a, b) in enumerate(pairs):
        want, strand = _best_strand(a, b, True)
        assert (_se(so[k]), so[k].strand) == (want, strand), k
        want, strand = _best_strand(a, b, False)
        for r in (al[k], ad[k]):
            assert ((r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.cigar or ""), r.strand) == (want, strand), k
        strands.append(strand)
    assert 0 < sum(strands) < len(strands)
    assert al[-2].strand == 0 and al[-2].score > 0 and al[-3].strand == 0


def test_band_height_tuning(sw):
    """The first batch of a shape times each int16x2 band height and keeps the
    fastest for that shape; tuned, cached and untuned calls return the same
    (oracle-equal) results."""
    c = sw.sw_ctx_create(0, workspace_bytes=2 << 30)
    try:
        pairs = _mixed_pairs(64, seed=71, lo=200, hi=2500)
        want = []
        for a, b in pairs:
            S, ei, ej = oracle.local_score(a, b)
            want.append((S, ei, ej) if S else (0, -1, -1))
        first = sw.sw_align_batch(c, pairs, flags=sw.SW_FLAG_SCORE_ONLY)
        again = sw.sw_align_batch(c, pairs, flags=sw.SW_FLAG_SCORE_ONLY)
        c.set_option(sw.SW_OPT_AUTOTUNE, 0)
        plain = sw.sw_align_batch(c, pairs, flags=sw.SW_FLAG_SCORE_ONLY)
        assert first[0].stats["tuned"] == 1 and again[0].stats["tuned"] == 0 and plain[0].stats["tuned"] == 0
        assert first[0].stats["band_rows"] in (256, 512, 1024)
        assert again[0].stats["band_rows"] == first[0].stats["band_rows"]
        for k, (a, b) in enumerate(pairs):
            got = [_se(r[k]) for r in (first, again, plain)]
            assert got[0] == got[1] == got[2] == want[k], k
    finally:
        c.close()


def test_tuning_table_export_import(sw):
    """The autotuner's table moves between contexts as text: a context that
    imports it runs the batch shape at the stored band height without timing
    it, with the same results; a table naming another GPU model or holding a
    malformed line is refused and changes nothing."""
    c1 = sw.sw_ctx_create(0, workspace_bytes=1 << 30)
    c2 = sw.sw_ctx_create(0, workspace_bytes=1 << 30)
    try:
        pairs = _mixed_pairs(64, seed=72, lo=200, hi=2500)
        first = sw.sw_align_batch(c1, pairs, flags=sw.SW_FLAG_SCORE_ONLY)
        assert first[0].stats["tuned"] == 1
        text = c1.tuning_export()
        lines = text.splitlines()
        assert lines[0].startswith("swgb-tuning 1 ") and len(lines) == 2
        for bad in (text.replace("swgb-tuning 1 ", "swgb-tuning 1 other "),
                    lines[0] + "\nzz 16\n", lines[0] + "\n1f 12\n"):
            with pytest.raises(sw.SwError):
                c2.tuning_import(bad)
        assert c2.tuning_export() == lines[0] + "\n"
        c2.tuning_import(text)
        assert c2.tuning_export() == text
        again = sw.sw_align_batch(c2, pairs, flags=sw.SW_FLAG_SCORE_ONLY)
        assert again[0].stats["tuned"] == 0
        assert again[0].stats["band_rows"] == first[0].stats["band_rows"]
        assert [_se(r) for r in again] == [_se(r) for r in first]
    finally:
        c1.close()
        c2.close()
