"""The checkpointable score pass (sw_score_job_*): the forward pass run in
segments of row bands, its state snapshotted to host memory and resumed in
another context.  Every result must equal the oracle's (score and end point)
and sw_score's, whatever the segment boundaries; a snapshot must be refused
for other sequences, another scheme or pruning flag, and when damaged.
"""
import numpy as np
import pytest

import oracle
from gen import synth

pytestmark = pytest.mark.gpu


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


def _se(r):
    return (r.score, r.a_end, r.b_end)


def _run_segments(job, sizes):
    for k in sizes:
        job.run(k)
    return job.run(-1)


def test_segments_equal_oracle(sw, ctx):
    a, b0 = synth.related_pair(21_000, seed=601)
    a, b = a[:20_500], b0[:18_300]
    want = oracle.local_score(a, b)
    for flags in (0, sw.SW_FLAG_NO_PRUNE):
        job = sw.sw_score_job_create(ctx, a, b, flags=flags)
        try:
            done, total = _run_segments(job, [1, 7, 13, 2])
            assert done == total > 20
            r = job.result()
        finally:
            job.close()
        assert _se(r) == want
        assert _se(sw.sw_score(ctx, a, b, flags=flags)) == want


def test_snapshot_resume_in_another_context(sw, ctx):
    a, b0 = synth.related_pair(300_000, seed=602)
    a, b = a, b0[:250_000]
    want = _se(sw.sw_score(ctx, a, b))
    job = sw.sw_score_job_create(ctx, a, b)
    try:
        assert job.wave_bands > 0 and job.bands_total > 400
        first = job.snapshot()                       # before any band ran
        done, total = job.run(400)
        mid = job.snapshot()
        with pytest.raises(sw.SwError) as e:
            job.result()                             # bands left
        assert e.value.status == sw.SW_EPENDING
    finally:
        job.close()
    assert 0 < done < total
    c2 = sw.sw_ctx_create(0, workspace_bytes=1 << 30)
    try:
        for snap, segs in ((mid, [300]), (mid, []), (first, [total // 2])):
            j2 = sw.sw_score_job_resume(c2, a, b, snap)
            try:
                d2, t2 = _run_segments(j2, segs)
                assert d2 == t2 == total
                assert _se(j2.result()) == want
            finally:
                j2.close()
    finally:
        c2.close()


def test_resume_refuses_other_inputs_and_damage(sw, ctx):
    a, b0 = synth.related_pair(30_000, seed=603)
    a, b = a, b0[:20_000]
    job = sw.sw_score_job_create(ctx, a, b)
    try:
        job.run(20)
        snap = job.snapshot()
    finally:
        job.close()
    b2 = b.copy()
    b2[12_345] = (b2[12_345] + 1) % 4          # one base differs
    bad = [
        dict(a=a, b=b2, snapshot=snap),                                          # other sequence
        dict(a=a, b=b, snapshot=snap, scheme=sw.Scheme(1, -3, 6, 2)),           # other scheme
        dict(a=a, b=b, snapshot=snap, flags=sw.SW_FLAG_NO_PRUNE),               # other pruning flag
        dict(a=a, b=b, snapshot=b"XXXX" + snap[4:]),                             # damaged magic
        dict(a=a, b=b, snapshot=snap[:-16]),                                     # truncated
        dict(a=a[:-1], b=b, snapshot=snap),                                      # other length
    ]
    for k, kw in enumerate(bad):
        try:
            sw.sw_score_job_resume(ctx, **kw).close()
            status = sw.SW_OK
        except sw.SwError as e:
            status = e.status
        assert status == sw.SW_EINVAL, k
    j = sw.sw_score_job_resume(ctx, a, b, snap)                                 # the right inputs work
    try:
        assert j.run(0)[0] == 20                  # progress only
        j.run(-1)
        assert _se(j.result()) == oracle.local_score(a, b)
    finally:
        j.close()


def test_int32_lanes_and_device_inputs(sw, ctx):
    import torch
    a, b0 = synth.related_pair(12_000, seed=604)
    a, b = a[:11_111], b0[:9_999]
    want = oracle.local_score(a, b)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    ctx.set_option(sw.SW_OPT_FORWARD_LANES, 32)
    try:
        job = sw.sw_score_job_create(ctx, ta, tb)
        try:
            job.run(3)
            snap = job.snapshot()
        finally:
            job.close()
        j2 = sw.sw_score_job_resume(ctx, ta, tb, snap)
        try:
            j2.run(-1)
            r = j2.result()
        finally:
            j2.close()
    finally:
        ctx.set_option(sw.SW_OPT_FORWARD_LANES, 0)
    assert r.stats["band_rows"] % 32 == 0 and _se(r) == want


def test_one_cta_per_sm_segments(sw, ctx):
    """Segments long enough for the one-CTA-per-SM layout, then a short one,
    with a snapshot and resume between them, on the planted pair of the
    full-width layout test."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 2 * sms * 20 * 256 + 70_001
    st = synth.Rng(97).stream()
    a = synth.random_bases(st, n)
    core = a[n - 300_000:n - 299_400].copy()
    b = np.concatenate([synth.random_bases(st, 50), synth.mutate(st, core), synth.random_bases(st, 40)])
    ctx.set_option(sw.SW_OPT_FORWARD_LANES, 16)
    ctx.set_option(sw.SW_OPT_ROWS_PER_THREAD, 4)
    try:
        want = _se(sw.sw_score(ctx, a, b))
        job = sw.sw_score_job_create(ctx, a, b)
        try:
            done, total = job.run(2 * sms * 20 + 3)
            snap = job.snapshot()
        finally:
            job.close()
        j2 = sw.sw_score_job_resume(ctx, a, b, snap)
        try:
            assert j2.run(-1) == (total, total)
            r = j2.result()
        finally:
            j2.close()
    finally:
        ctx.set_option(sw.SW_OPT_FORWARD_LANES, 0)
        ctx.set_option(sw.SW_OPT_ROWS_PER_THREAD, 0)
    assert 0 < done < total and r.stats["band_rows"] == 256
    assert _se(r) == want and want[0] > 0
