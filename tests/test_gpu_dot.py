"""mw_dot_batched: m-double inner products (Section 2's s_i of one inner
product; Table 2 times 1,024 of them of length 6,144).

Every inner product equals the oracle's error-free summation with the same
plan (24-bit digits) bit for bit, and meets the bound 2K 2^(-52m) sum |a||b|
against the exact rational inner product."""
import numpy as np
import pytest
import torch

from conftest import record_worst, to_dev
from oracle import exact, slicing
from synthetic import SplitMix64, loguniform_mdouble, paper_pattern_mdouble, uniform_mdouble

pytestmark = pytest.mark.gpu


def operands(kind, rng, m, count, K):
    if kind == "uniform":
        return uniform_mdouble(rng, m, count, K), uniform_mdouble(rng, m, count, K)
    if kind == "loguniform":
        return (loguniform_mdouble(rng, m, count, K, -20, 20),
                loguniform_mdouble(rng, m, count, K, -20, 20))
    return paper_pattern_mdouble(rng, m, count, K), paper_pattern_mdouble(rng, m, count, K)


def check_dots(mw, cuda, A, B, rows=None, name=None):
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_dot(tA, tB)
    C = mw.mw_dot_batched(tA, tB, plan).cpu().numpy()
    m, count, K = A.shape
    worst = 0.0
    for i in (range(count) if rows is None else rows):
        a = A[:, i:i + 1, :]
        b = np.ascontiguousarray(B[:, i:i + 1, :].transpose(0, 2, 1))
        sp = slicing.SlicedProduct(a, b, plan.w, plan.S_A, plan.S_B, plan.D)
        assert sp.A.in_range and sp.B.in_range
        got = C[:, i].reshape(m, 1, 1)
        assert np.array_equal(got, sp.result()), i
        worst = max(worst, exact.ExactProduct(a, b, [0], [0]).error_ratio(got).max())
    assert worst <= 1.0
    if name:
        record_worst(name, worst)
    return C, plan


@pytest.mark.parametrize("m", [2, 4, 8])
@pytest.mark.parametrize("count,K,kind", [
    (6, 1, "uniform"), (9, 300, "loguniform"), (3, 2000, "uniform"), (4, 6144, "pattern"),
    (2, 257, "pattern"),
])
def test_dot_bit_exact(mw, cuda, m, count, K, kind):
    rng = SplitMix64(700 + 10 * m + K)
    A, B = operands(kind, rng, m, count, K)
    check_dots(mw, cuda, A, B)


@pytest.mark.parametrize("count,K,kind", [(4, 1, "uniform"), (3, 40, "pattern"), (2, 700, "pattern")])
def test_dot_hexa_double(mw, cuda, count, K, kind):
    """m = 16 inner products (35 or 36 digits of 24 bits a term)."""
    rng = SplitMix64(760 + K)
    A, B = operands(kind, rng, 16, count, K)
    check_dots(mw, cuda, A, B)


@pytest.mark.parametrize("m", [2, 4, 8, 16])
def test_dot_words_not_normalised(mw, cuda, m):
    """Entries whose later word is larger than the first (input that is not
    normalised): the shared exponent is still ilogb + 1 of the largest word of
    any entry, so the vectors are cut again with it; bit-exact vs the oracle."""
    rng = SplitMix64(770 + m)
    A, B = operands("uniform", rng, m, 3, 50)
    A[0, 1, 7] = 0.0
    A[1, 1, 7] = 4.0                    # leading word zero, the second 4
    A[0, 2, 3] = 1e-3
    A[m - 1, 2, 3] = 8.0                # the last word far above the first
    B[0, 0, 9] = 0.0
    B[1, 0, 9] = -16.0
    check_dots(mw, cuda, A, B)


def test_dot_edge_cases(mw, cuda):
    """Zero vectors, one nonzero entry, exact cancellation, a tie."""
    m, K = 4, 5
    A = np.zeros((m, 4, K))
    B = np.zeros((m, 4, K))
    B[0, 0, :] = 1.0                                   # 0: a = 0
    A[0, 1, 2] = 3.0; B[0, 1, 2] = -0.5                # 1: one product, -1.5
    A[0, 2, :2] = [1.0, 1.0]; B[0, 2, :2] = [2.0 ** 40, -2.0 ** 40]   # 2: cancels to 0
    A[0, 3, :2] = [1.0, 2.0 ** -53]; B[0, 3, :2] = [1.0, 1.0]          # 3: 1 + 2^-53, a tie
    C, _ = check_dots(mw, cuda, A, B)
    assert list(C[:, 0]) == [0.0] * m
    assert list(C[:, 1]) == [-1.5, 0.0, 0.0, 0.0]
    assert list(C[:, 2]) == [0.0] * m
    assert list(C[:, 3]) == [1.0, 2.0 ** -53, 0.0, 0.0]


def test_dot_strided_rows(mw, cuda):
    """Rows of a larger matrix (lda > K) and a result into a wider tensor."""
    rng = SplitMix64(720)
    A, B = operands("uniform", rng, 2, 5, 200)
    tA = to_dev(A, cuda)[:, :, :150]
    tB = to_dev(B, cuda)[:, :, :150]
    plan = mw.plan_dot(tA, tB)
    C = mw.mw_dot_batched(tA, tB, plan).cpu().numpy()
    sub_A = np.ascontiguousarray(A[:, :, :150])
    sub_B = np.ascontiguousarray(B[:, :, :150])
    for i in range(5):
        sp = slicing.SlicedProduct(sub_A[:, i:i + 1], np.ascontiguousarray(
            sub_B[:, i:i + 1].transpose(0, 2, 1)), plan.w, plan.S_A, plan.S_B, plan.D)
        assert np.array_equal(C[:, i].reshape(2, 1, 1), sp.result())


@pytest.mark.slow
@pytest.mark.parametrize("m", [2, 4, 8, 16])
def test_table2_workload(mw, cuda, m):
    """1,024 inner products of length 6,144 on the Section 2 bit pattern
    (Table 2's workload), 16 sampled products against the oracle."""
    from synthetic import table2_operands
    A, B = table2_operands(m)
    rows = [int(i) for i in SplitMix64(730).next(16) % np.uint64(A.shape[1])]
    check_dots(mw, cuda, A, B, rows=rows, name=f"table 2 workload m={m}, 16 inner products")


def test_dot_rejects_bad_plans(mw, cuda):
    rng = SplitMix64(740)
    A, B = operands("uniform", rng, 2, 2, 10)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    gemm_plan = mw.plan_for(tA, tB, "ozaki", False, True)
    with pytest.raises(mw.MWError):
        mw.mw_dot_batched(tA, tB, gemm_plan)
    plan = mw.plan_dot(tA, tB)
    plan.S_A = plan.S_B = 40                          # not compiled
    with pytest.raises(mw.MWError):
        mw.mw_dot_batched(tA, tB, plan)


def test_dot_status_bits(mw, cuda):
    """Non-finite input raises MW_ENONFINITE, a spread beyond the plan's raises
    the MW_WRANGE warning, a clean call raises nothing."""
    mw.get_status(clear=True)
    rng = SplitMix64(750)
    A, B = operands("uniform", rng, 2, 3, 40)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_dot(tA, tB)
    mw.mw_dot_batched(tA, tB, plan, check=False)
    assert mw.get_status(clear=True) == 0
    A2 = A.copy()
    A2[0, 1, 7] = np.nan
    mw.mw_dot_batched(to_dev(A2, cuda), tB, plan, check=False)
    assert mw.get_status(clear=True) & mw.MW_ENONFINITE
    A3 = A.copy()
    A3[:, 2, 5] *= 2.0 ** -40                       # spread of row 2 beyond the plan's
    mw.mw_dot_batched(to_dev(A3, cuda), tB, plan, check=False)
    assert mw.get_status(clear=True) & mw.MW_WRANGE
