"""mw_convolve_batched: products of truncated m-double power series (Section 1's
application; Section 2's diagonal sums s_i are these convolutions).  Every
coefficient equals the oracle's error-free summation of its inner product
(a_0..a_i against b_i..b_0) with the same plan bit for bit, and meets its bound
2 (i+1) 2^(-52m) sum |a_k||b_(i-k)| against the exact convolution."""
from fractions import Fraction

import numpy as np
import pytest
import torch

from conftest import record_worst, to_dev
from oracle import exact, series
from synthetic import SplitMix64, loguniform_mdouble, paper_pattern_mdouble, uniform_mdouble

pytestmark = pytest.mark.gpu


def check_series(mw, cuda, A, B, rows=None, label=None):
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_convolve(tA, tB)
    C = mw.mw_convolve_batched(tA, tB, plan).cpu().numpy()
    m, count, n = A.shape
    worst = 0.0
    for s in (range(count) if rows is None else rows):
        a, b = A[:, s, :], B[:, s, :]
        want = series.convolution_sliced(a, b, plan.w, plan.S_A, plan.D)
        assert np.array_equal(C[:, s, :], want), s
        ex, bd = series.convolution_exact(a, b), series.convolution_bound(a, b)
        for i in range(n):
            err = abs(exact.to_fraction(C[:, s, i]) - ex[i])
            assert err <= bd[i], (s, i)
            if bd[i]:
                worst = max(worst, float(err / bd[i]))
    if label:
        record_worst(label, worst)
    return C


@pytest.mark.parametrize("m", [2, 4, 8, 16])
def test_series_products_bit_exact(mw, cuda, m):
    rng = SplitMix64(1200 + m)
    A, B = uniform_mdouble(rng, m, 5, 40), uniform_mdouble(rng, m, 5, 40)
    check_series(mw, cuda, A, B, label=f"series m={m}, 5 x 40 coefficients")


@pytest.mark.parametrize("kind,n", [("loguniform", 129), ("pattern", 300), ("uniform", 1)])
def test_series_lengths_and_ranges(mw, cuda, kind, n):
    """Degrees past one CTA's 256 threads, a single coefficient, wide ranges and the
    Section 2 bit pattern."""
    rng = SplitMix64(1210 + n)
    if kind == "loguniform":
        A, B = loguniform_mdouble(rng, 4, 3, n, -10, 10), loguniform_mdouble(rng, 4, 3, n, -10, 10)
    elif kind == "pattern":
        A, B = paper_pattern_mdouble(rng, 2, 2, n), paper_pattern_mdouble(rng, 2, 2, n)
    else:
        A, B = uniform_mdouble(rng, 8, 4, n), uniform_mdouble(rng, 8, 4, n)
    check_series(mw, cuda, A, B, rows=None if n < 200 else [0, 1])


def test_series_closed_forms(mw, cuda):
    """(1 - x) times the geometric series is 1; the geometric series squared has
    coefficients i + 1 (exact in every word)."""
    m, n = 4, 64
    def words(vals):
        return np.array([exact.greedy_words(Fraction(v), m) for v in vals]).T.copy()[:, None, :]
    one_minus_x = words([1, -1] + [0] * (n - 2))
    geometric = words([1] * n)
    C = mw.mw_convolve_batched(to_dev(one_minus_x, cuda), to_dev(geometric, cuda)).cpu().numpy()
    assert np.array_equal(C, words([1] + [0] * (n - 1)))
    C = mw.mw_convolve_batched(to_dev(geometric, cuda), to_dev(geometric, cuda)).cpu().numpy()
    assert np.array_equal(C, words([i + 1 for i in range(n)]))


def test_series_strided_output_and_rejects(mw, cuda):
    """Series in wider rows (ld > n) and a bad plan or shape raise."""
    rng = SplitMix64(1230)
    A, B = uniform_mdouble(rng, 2, 3, 50), uniform_mdouble(rng, 2, 3, 50)
    tA, tB = to_dev(A, cuda)[:, :, :37], to_dev(B, cuda)[:, :, :37]
    plan = mw.plan_convolve(tA, tB)
    Cw = torch.zeros((2, 3, 45), dtype=torch.float64, device=cuda)
    mw.mw_convolve_batched(tA, tB, plan, C=Cw[:, :, :37])
    for s in range(3):
        want = series.convolution_sliced(A[:, s, :37], B[:, s, :37], plan.w, plan.S_A, plan.D)
        assert np.array_equal(Cw[:, s, :37].cpu().numpy(), want)
    assert not Cw[:, :, 37:].any()
    with pytest.raises(mw.MWError):
        mw.mw_convolve_batched(tA, tB, mw.mw_plan_gemm(2, "ozaki", 3, 3, 37, 0, 0))
    with pytest.raises(mw.MWError):
        mw.mw_convolve_batched(tA, tB[:, :2, :], plan)
