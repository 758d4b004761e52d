"""sw_score_static: the allocation-free forward pass.

Some callers cannot allocate device memory when they need a score (their
framework reserves all device memory up front, or their hot path forbids
cudaMalloc/cudaFree).  sw_score_static takes its scratch from a library-wide
static device array instead.  It must give exactly what sw_score gives, on two
calls in a row (the second call must not see the first call's leftovers), and
must refuse inputs larger than its static scratch.  This file sorts last so a
failure here does not hide the other tests' results.
"""
import ctypes

import numpy as np
import pytest

from gen import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import paper_1304_5966_gb300 as m
    from paper_1304_5966_gb300 import build
    build.build()
    return m


def _c_abi_call(sw, ta, tb, scheme=None):
    """Call the C entry point directly through ctypes."""
    import torch
    L = sw.lib()
    sch, keep = (scheme or sw.DNA)._c()
    res = sw._Result()
    st = L.sw_score_static(ctypes.c_void_p(ta.data_ptr()), ta.numel(), ctypes.c_void_p(tb.data_ptr()),
                           tb.numel(), ctypes.byref(sch),
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(res))
    return st, res


def test_static_scratch_matches_sw_score_twice(sw):
    import torch
    ctx = sw.sw_ctx_create(0, workspace_bytes=256 << 20)
    try:
        cases = [synth.related_pair(60_000, seed=901), synth.random_pair(3_000, 45_000, seed=902)]
        for a, b in cases:                       # two calls in a row, different sizes and content
            ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
            st, res = _c_abi_call(sw, ta, tb)
            assert st == sw.SW_OK
            want = sw.sw_score(ctx, ta, tb)
            assert (res.score, res.a_end, res.b_end) == (want.score, want.a_end, want.b_end)
            assert res.score > 0
    finally:
        ctx.close()


def test_static_scratch_limits_and_codes(sw):
    import torch
    tb = torch.zeros(1_048_577, dtype=torch.uint8, device="cuda")
    ta = torch.zeros(10, dtype=torch.uint8, device="cuda")
    st, _ = _c_abi_call(sw, ta, tb)
    assert st == sw.SW_ENOMEM                    # beyond the static scratch
    bad = torch.tensor([0, 1, 7], dtype=torch.uint8, device="cuda")
    st, _ = _c_abi_call(sw, bad, bad)
    assert st == sw.SW_EINVAL                    # code >= alphabet
    # the binding wrapper gives the same numbers as the raw call
    a, b = synth.related_pair(5_000, seed=903)
    ta2, tb2 = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    r = sw.sw_score_static(ta2, tb2)
    st, res = _c_abi_call(sw, ta2, tb2)
    assert st == sw.SW_OK and (r.score, r.a_end, r.b_end) == (res.score, res.a_end, res.b_end)
