"""Serving loop (sw_server_*): continuous batching.

Requests of mixed sizes and kinds arrive while earlier ones run; every result
must equal the same request run alone (and the oracle on a sample); admission
refuses what cannot fit the memory budget; queued requests can be cancelled.
"""
import threading
import time

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


def _requests(count, seed, lo=300, hi=20_000):
    st = synth.Rng(seed).stream()
    lens = synth.log_uniform_int(st, lo, hi, count)
    kinds = st.below(count, 100)
    out = []
    for k in range(count):
        a, b = synth.related_pair(int(lens[k]), seed=seed * 7919 + k)
        out.append((a, b, bool(kinds[k] < 70)))
    return out


def _key(r):
    return (r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.cigar or "")


def test_mixed_stream_equals_alone(sw):
    ctx = sw.sw_ctx_create(0, workspace_bytes=6 << 30)
    alone_ctx = sw.sw_ctx_create(0, workspace_bytes=2 << 30)
    srv = sw.Server(ctx, workers=3)
    reqs = _requests(36, 1)
    tickets = [None] * len(reqs)

    def producer():
        for k, (a, b, so) in enumerate(reqs):
            tickets[k] = srv.submit(a, b, score_only=so)
            time.sleep(0.002 * (k % 5))          # staggered arrivals

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    got = [srv.poll(t) for t in tickets]
    srv.close()
    for k, ((a, b, so), r) in enumerate(zip(reqs, got)):
        if so:
            w = sw.sw_score(alone_ctx, a, b)
            assert (r.score, r.a_end, r.b_end) == (w.score, w.a_end, w.b_end), k
        else:
            w = sw.sw_align(alone_ctx, a, b)
            assert _key(r) == _key(w), k
    for k in (0, 5, 11):
        a, b, so = reqs[k]
        o = oracle.align(a, b)
        assert got[k].score == o.score and got[k].a_end == o.a_end and got[k].b_end == o.b_end
        if not so:
            assert _key(got[k]) == (o.score, o.a_begin, o.a_end, o.b_begin, o.b_end, o.cigar)
    ctx.close()
    alone_ctx.close()


def test_admission_and_cancel(sw):
    ctx = sw.sw_ctx_create(0, workspace_bytes=1 << 30)
    srv = sw.Server(ctx, workers=1, device_budget=64 << 20)
    big = np.zeros(3_000_000, np.uint8)
    with pytest.raises(sw.SwError) as e:
        srv.submit(big, big)                      # footprint beyond the worker's slice
    assert e.value.status == sw.SW_EBUSY
    reqs = _requests(12, 2, lo=8_000, hi=12_000)
    ts = [srv.submit(a, b, score_only=True) for a, b, _ in reqs]
    st = srv.cancel(ts[-1])
    assert st in (sw.SW_OK, sw.SW_EBUSY)
    for t in ts[:-1]:
        assert srv.poll(t).score > 0
    if st == sw.SW_OK:
        with pytest.raises(sw.SwError):
            srv.poll(ts[-1], timeout_us=0)        # retired ticket
    else:
        assert srv.poll(ts[-1]).score > 0
    srv.close()
    ctx.close()
