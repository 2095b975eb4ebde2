"""mw_gemm_noalloc, the product for callers that cannot allocate device memory
(a plug-in inside a host program that owns all device memory through its own
pool may not call cudaMalloc).  It runs mw_gemm on a fixed per-device scratch
array; its results must equal those of mw_gemm with a caller-allocated
workspace, bit for bit as every Ozaki-form test here requires, on two calls in
a row that reuse the same scratch.  This file is collected last on purpose."""
import ctypes

import pytest
import torch

from conftest import to_dev
from synthetic import SplitMix64, loguniform_mdouble

pytestmark = pytest.mark.gpu


def call_noalloc(mw, plan, tA, tB, C):
    m, M, N, K = mw._dims(tA, tB, False, False)
    pa, lda, psa = mw._mat(tA, "A")
    pb, ldb, psb = mw._mat(tB, "B")
    pc, ldc, psc = mw._mat(C, "C")
    return mw._lib.mw_gemm_noalloc(ctypes.byref(plan), 0, 0, M, N, K, pa, lda, psa, pb, ldb,
                                   psb, pc, ldc, psc, mw._stream())


def test_noalloc_matches_gemm_on_two_calls_in_a_row(mw, cuda):
    cases = [(2, 100, 90, 130, 401), (4, 64, 70, 200, 402)]
    for m, M, N, K, seed in cases:
        rng = SplitMix64(seed)
        tA = to_dev(loguniform_mdouble(rng, m, M, K, -6, 6), cuda)
        tB = to_dev(loguniform_mdouble(rng, m, K, N, -6, 6), cuda)
        plan = mw.plan_for(tA, tB, "ozaki")
        ref = mw.mw_gemm(tA, tB, plan)
        C = torch.full_like(ref, float("nan"))
        rc = call_noalloc(mw, plan, tA, tB, C)
        assert rc == mw.MW_OK, mw._lib.mw_last_error().decode()
        mw.check_status()
        assert torch.equal(C, ref)


def test_noalloc_allocates_nothing(mw, cuda):
    """After one call on the device (which may load the library's module and
    with it the scratch array), two more calls leave the device's free memory
    and torch's allocations unchanged, and give the same words."""
    rng = SplitMix64(403)
    tA = to_dev(loguniform_mdouble(rng, 2, 90, 110, -6, 6), cuda)
    tB = to_dev(loguniform_mdouble(rng, 2, 110, 80, -6, 6), cuda)
    plan = mw.plan_for(tA, tB, "ozaki")
    ref = mw.mw_gemm(tA, tB, plan)
    C = torch.empty_like(ref)
    assert call_noalloc(mw, plan, tA, tB, C) == mw.MW_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        C.fill_(float("nan"))
        assert call_noalloc(mw, plan, tA, tB, C) == mw.MW_OK, mw._lib.mw_last_error().decode()
        torch.cuda.synchronize()
        assert torch.equal(C, ref)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    mw.check_status()


def test_noalloc_rejects_a_product_beyond_its_scratch(mw, cuda):
    n = 2048
    tA = torch.zeros((2, n, n), dtype=torch.float64, device=cuda)
    tB = torch.zeros((2, n, n), dtype=torch.float64, device=cuda)
    C = torch.zeros((2, n, n), dtype=torch.float64, device=cuda)
    plan = mw.mw_plan_gemm(2, "ozaki", n, n, n, 0, 0)
    rc = call_noalloc(mw, plan, tA, tB, C)
    assert rc == mw.MW_ENOSPC
    assert "scratch" in mw._lib.mw_last_error().decode()
    assert not C.any()
