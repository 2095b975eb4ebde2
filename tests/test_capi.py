"""The C interface on the CPU: the library loads, exports every entry point of
include/mw.h, rejects bad arguments on the host, and its planner's slice counts
meet the error bound when the oracle runs the method with them."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2606_20863_gb300", "libmw.so")


@pytest.fixture(scope="module")
def mw():
    if not os.path.exists(LIB):
        import __graft_entry__
        __graft_entry__.build()
    import paper_2606_20863_gb300 as mw
    return mw


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "mw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mw_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(mw):
    lib = ctypes.CDLL(LIB)
    names = declared_entry_points()
    assert "mw_gemm" in names and "mw_split" in names and "mw_gemm_backward" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(mw.EXPORTED) <= set(names)


def test_version(mw):
    assert "sm_103a" in mw.version()


@pytest.mark.parametrize("m,mode", [(2, "ozaki"), (4, "ozaki"), (8, "ozaki"), (16, "ozaki"),
                                    (2, "plain"), (4, "plain"), (8, "plain")])
def test_plan_constraints(mw, m, mode):
    for K in (1, 7, 64, 1024, 4096, 65536):
        for ra, rb in ((0, 0), (16, 16), (40, 40), (3, 60)):
            p = mw.mw_plan_gemm(m, mode, 100, 100, K, ra, rb)
            lgK = math.log2(K)
            # truncation of each operand within a quarter of the budget
            assert p.w * p.S_A >= 52 * m + ra + math.log2(m) + 5 - lgK - 1e-9
            assert p.w * p.S_B >= 52 * m + rb + math.log2(m) + 5 - lgK - 1e-9
            S_min = min(p.S_A, p.S_B)
            if p.D < p.S_A + p.S_B - 1:
                assert p.w * p.D >= 52 * m + ra + rb + math.log2(S_min) + 6 - lgK - 1e-9
            if mode == "ozaki":
                assert p.w == 8 and p.chunk * 2 ** (2 * p.w - 2) <= 2 ** 24
                max_s = S_min * K * 2 ** (2 * p.w - 2)
                assert max_s * 2 ** (p.w * (p.group - 1)) * (1 + 2 ** (1 - p.w)) < 2 ** 63
            else:
                assert S_min * K * 2 ** (2 * p.w - 2) <= 2 ** 53


@pytest.mark.parametrize("m", [2, 4, 8, 16])
def test_dot_plan_constraints(mw, m):
    """MW_DOT plans: 24-bit digits, S_A = S_B within the compiled range, the
    same truncation budget as products, D <= S + 4, a thread's int64 sums
    (ceil(K/256) products below 2^46) safe; too long or too wide is refused."""
    lo, hi = {2: (4, 8), 4: (8, 12), 8: (17, 21), 16: (35, 36)}[m]
    spreads = ((0, 0), (16, 16)) if m == 16 else ((0, 0), (16, 16), (40, 40), (3, 60))
    for K in (1, 7, 700, 6144, 100000):
        for ra, rb in spreads:
            p = mw.mw_plan_gemm(m, "dot", 1, 1, K, ra, rb)
            lgK = math.log2(K)
            assert p.w == 24 and p.S_A == p.S_B and lo <= p.S_A <= hi
            assert p.w * p.S_A >= 52 * m + max(ra, rb) + math.log2(m) + 5 - lgK - 1e-9
            if p.D < 2 * p.S_A - 1:
                assert p.w * p.D >= 52 * m + ra + rb + math.log2(p.S_A) + 6 - lgK - 1e-9
            assert p.D <= p.S_A + 4
            assert p.S_A * math.ceil(K / 256) * 2 ** 46 < 2 ** 63
    with pytest.raises(mw.MWError):
        mw.mw_plan_gemm(m, "dot", 1, 1, 10 ** 8, 0, 0)        # K too long for int64 sums
    with pytest.raises(mw.MWError):
        mw.mw_plan_gemm(m, "dot", 1, 1, 100, 300, 300)        # spreads need too many pieces
    with pytest.raises(mw.MWError):
        mw.mw_plan_gemm(m, "dot", 4, 1, 100, 0, 0)            # one inner product per plan


@pytest.mark.parametrize("m,lo,hi", [(2, -6, 6), (4, -20, 20), (8, -3, 3), (16, -2, 2)])
def test_dot_planner_meets_bound_on_the_oracle(mw, m, lo, hi):
    """The MW_DOT plan from the measured spreads keeps the oracle's summation
    with 24-bit digits within the bound (one inner product of length 500)."""
    from oracle import exact, slicing
    from synthetic import SplitMix64, loguniform_mdouble
    rng = SplitMix64(95 + m)
    a = loguniform_mdouble(rng, m, 1, 500, lo, hi)
    b = loguniform_mdouble(rng, m, 500, 1, lo, hi)
    ra = int(slicing.row_exponents(a)[1].max())
    rb = int(slicing.row_exponents(slicing.logical(b, True))[1].max())
    p = mw.mw_plan_gemm(m, "dot", 1, 1, 500, ra, rb)
    sp = slicing.SlicedProduct(a, b, p.w, p.S_A, p.S_B, p.D)
    assert sp.A.in_range and sp.B.in_range
    assert exact.exact_product_full(a, b).error_ratio(sp.result()).max() <= 1.0


def test_hexa_double_forms(mw):
    """m = 16 plans in the tensor-core form and for inner products, not in the
    FP64 form."""
    assert mw.mw_plan_gemm(16, "ozaki", 100, 100, 1024, 0, 0).S_A >= 104
    with pytest.raises(mw.MWError):
        mw.mw_plan_gemm(16, "plain", 100, 100, 1024, 0, 0)


def test_host_side_errors(mw):
    with pytest.raises(mw.MWError):
        mw.mw_plan_gemm(3, "ozaki", 10, 10, 10, 0, 0)
    with pytest.raises(mw.MWError):
        mw.mw_plan_gemm(2, "ozaki", 0, 10, 10, 0, 0)
    with pytest.raises(mw.MWError):
        mw.mw_plan_gemm(2, "ozaki", 10, 10, 10, -1, 0)
    p = mw.mw_plan_gemm(2, "ozaki", 64, 64, 64, 0, 0)
    p.group = 99
    with pytest.raises(mw.MWError):
        mw.workspace_size(p, 64, 64, 64)
    p = mw.mw_plan_gemm(2, "plain", 64, 64, 64, 0, 0)
    p.w = 26
    with pytest.raises(mw.MWError):           # FP64 sums no longer exact
        mw.workspace_size(p, 64, 64, 64)
    # a NULL operand is refused before any GPU work
    p = mw.mw_plan_gemm(2, "ozaki", 8, 8, 8, 0, 0)
    rc = mw._lib.mw_gemm(ctypes.byref(p), 0, 0, 8, 8, 8, None, 8, 64, None, 8, 64, None, 8, 64,
                         None, 0, None)
    assert rc == mw.MW_EINVAL
    assert "NULL" in mw._lib.mw_last_error().decode()


def test_workspace_layout_is_consistent(mw):
    p = mw.mw_plan_gemm(4, "ozaki", 300, 200, 1000, 10, 10)
    off, total = mw.workspace_layout(p, 300, 200, 1000)
    Kp = 1024
    assert off[0] == 0 and off[1] >= 4 * (2 * 300 + 2 * 200 + 2)
    assert off[2] - off[1] >= p.S_A * 300 * Kp * 2
    assert off[3] - off[2] >= p.S_B * 200 * Kp * 2
    G = -(-p.D // p.group)
    assert total - off[3] >= G * 300 * 200 * 8
    assert total == mw.workspace_size(p, 300, 200, 1000)
    assert all(o % 256 == 0 for o in off)


@pytest.mark.parametrize("m,mode,lo,hi", [(2, "ozaki", -20, 20), (2, "plain", -8, 8),
                                          (4, "ozaki", -8, 8), (8, "ozaki", -4, 4),
                                          (16, "ozaki", -2, 2)])
def test_planner_meets_bound_on_the_oracle(mw, m, mode, lo, hi):
    """The plan computed from the measured spreads gives errors within the bound
    when the CPU oracle carries out the method with it, including operands
    built so that small entries of A meet large entries of B."""
    from oracle import exact, slicing
    from synthetic import SplitMix64, loguniform_mdouble
    rng = SplitMix64(90 + m)
    n = 20
    A = loguniform_mdouble(rng, m, n, n, lo, hi)
    B = loguniform_mdouble(rng, m, n, n, lo, hi)
    # adversarial: row 0 of A tiny except one huge entry; column 0 of B the mirror
    A[:, 0, 1:] *= 2.0 ** (lo - hi)
    A[:, 0, 0] = loguniform_mdouble(rng, m, 1, 1, hi - 1, hi)[:, 0, 0]
    B[:, 0, 0] *= 2.0 ** (lo - hi)
    ra = int(slicing.row_exponents(A)[1].max())
    rb = int(slicing.row_exponents(slicing.logical(B, True))[1].max())
    p = mw.mw_plan_gemm(m, mode, n, n, n, ra, rb)
    sp = slicing.SlicedProduct(A, B, p.w, p.S_A, p.S_B, p.D)
    assert sp.A.in_range and sp.B.in_range
    ratio = exact.exact_product_full(A, B).error_ratio(sp.result())
    assert ratio.max() <= 1.0


# ---- batches, host side (no GPU memory is touched) --------------------------------------

def _describe(mw, shapes):
    arr = np.ascontiguousarray(np.array(shapes, dtype=np.int64).reshape(-1, 3))
    b = mw.mw_batch()
    rc = mw._lib.mw_batch_describe(len(shapes), arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   ctypes.byref(b))
    return rc, b


def _ozaki_plan(mw, m, S=56, D=60):
    p = mw.mw_plan()
    p.m, p.mode, p.w, p.S_A, p.S_B, p.D, p.group, p.chunk = m, mw.MW_OZAKI, 8, S, S, D, 5, 256
    p.range_A = p.range_B = -1
    return p


def test_batch_describe_sums(mw):
    rc, b = _describe(mw, [(3, 5, 7), (128, 1, 64), (1, 90, 2)])
    assert rc == mw.MW_OK
    assert (b.count, b.sum_M, b.sum_N, b.sum_MN) == (3, 132, 96, 3 * 5 + 128 + 90)
    assert (b.max_M, b.max_N, b.min_K, b.max_K) == (128, 90, 2, 64)
    rc, _ = _describe(mw, [(3, 0, 7)])
    assert rc == mw.MW_EINVAL


def test_batch_workspace_grows_and_takes_hexa_doubles(mw):
    small, big = _describe(mw, [(8, 8, 8)] * 10)[1], _describe(mw, [(100, 100, 100)] * 10)[1]
    size_s, size_b = ctypes.c_size_t(0), ctypes.c_size_t(0)
    p = _ozaki_plan(mw, 8)
    assert mw._lib.mw_gemm_batched_workspace_size(ctypes.byref(p), ctypes.byref(small),
                                                  ctypes.byref(size_s)) == mw.MW_OK
    assert mw._lib.mw_gemm_batched_workspace_size(ctypes.byref(p), ctypes.byref(big),
                                                  ctypes.byref(size_b)) == mw.MW_OK
    # the 100^3 problems at least hold their pieces: S bf16 planes of 100 x 128 per operand
    assert size_b.value > size_s.value and size_b.value >= 2 * 10 * 56 * 100 * 128 * 2
    p16 = _ozaki_plan(mw, 16, S=112, D=116)
    assert mw._lib.mw_gemm_batched_workspace_size(ctypes.byref(p16), ctypes.byref(small),
                                                  ctypes.byref(size_s)) == mw.MW_OK
    assert size_s.value >= 2 * 10 * 8 * 112 * 8 * 2       # 112 slices of every 8 x 8 problem
    p3 = _ozaki_plan(mw, 8)
    p3.m = 3
    assert mw._lib.mw_gemm_batched_workspace_size(ctypes.byref(p3), ctypes.byref(small),
                                                  ctypes.byref(size_s)) == mw.MW_EINVAL


def test_batch_spread_workspace_bound(mw):
    """mw_measure_spread_batched: its workspace size stays within the bound the
    header states, and one byte less fails with MW_ENOSPC on the host before any
    GPU work (no GPU memory is touched)."""
    for shapes in ([(8, 8, 8)], [(int(n), int(n), int(n)) for n in (8, 77, 128, 33)],
                   [(1, 3000, 5), (700, 1, 2)] * 50, [(128, 128, 128)] * 2000):
        _, b = _describe(mw, shapes)
        size = ctypes.c_size_t(0)
        assert mw._lib.mw_measure_spread_batched_workspace_size(
            8, ctypes.byref(b), ctypes.byref(size)) == mw.MW_OK
        bound = 8192 + 256 * b.count + 16 * (b.sum_M + b.sum_N) + b.sum_MN // 32
        assert 0 < size.value <= bound
        ra, rb = ctypes.c_int(0), ctypes.c_int(0)
        fake = ctypes.c_void_p(0x1000)       # never dereferenced: the size check comes first
        rc = mw._lib.mw_measure_spread_batched(8, ctypes.byref(b), fake, fake, size.value - 1,
                                               ctypes.byref(ra), ctypes.byref(rb), None)
        assert rc == mw.MW_ENOSPC
        rc = mw._lib.mw_measure_spread_batched(8, ctypes.byref(b), fake, None, size.value,
                                               ctypes.byref(ra), ctypes.byref(rb), None)
        assert rc == mw.MW_ENOSPC
    size = ctypes.c_size_t(0)
    assert mw._lib.mw_measure_spread_batched_workspace_size(
        3, ctypes.byref(b), ctypes.byref(size)) == mw.MW_EINVAL


def test_elementwise_rejects_bad_arguments(mw):
    """mw_elementwise checks op, m, n, pointers and strides on the host, before
    any device work; n = 0 does nothing."""
    f = mw._lib.mw_elementwise
    p = ctypes.c_void_p(4096)                 # never dereferenced: every call below fails first
    assert f(3, 2, 10, p, 10, p, 10, p, 10, None) == mw.MW_EINVAL
    assert f(0, 3, 10, p, 10, p, 10, p, 10, None) == mw.MW_EINVAL
    assert f(0, 16, 10, p, 10, p, 10, p, 10, None) == mw.MW_EINVAL
    assert f(2, 2, -1, p, 10, p, 10, p, 10, None) == mw.MW_EINVAL
    assert f(1, 4, 10, None, 10, p, 10, p, 10, None) == mw.MW_EINVAL
    assert f(1, 4, 10, p, 9, p, 10, p, 10, None) == mw.MW_EINVAL
    assert "stride" in mw._lib.mw_last_error().decode()
    assert f(2, 8, 0, None, 0, None, 0, None, 0, None) == mw.MW_OK
