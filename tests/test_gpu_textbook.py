"""MW_TEXTBOOK: the "ordinary" m-double product (Table 2's comparison) on the
GPU.  Its words equal the CPU oracle's textbook product (the same error-free
transformations in the same order, k ascending) bit for bit, for m = 2, 4, 8,
both orientations of each operand and ragged tiles; and meet the bound against
the exact product."""
import numpy as np
import pytest

from conftest import record_worst, to_dev
from oracle import exact, textbook
from synthetic import SplitMix64, loguniform_mdouble, uniform_mdouble

pytestmark = pytest.mark.gpu


def logical(X, trans):
    return np.ascontiguousarray(X.transpose(0, 2, 1)) if trans else X


@pytest.mark.parametrize("m,M,N,K,lo", [
    (2, 37, 45, 50, None), (4, 33, 17, 70, -8), (8, 20, 19, 40, None), (2, 1, 1, 1, -3),
    (4, 70, 35, 129, -20),
])
def test_textbook_bit_exact_vs_oracle(mw, cuda, m, M, N, K, lo):
    rng = SplitMix64(1300 + m + M)
    if lo is None:
        A, B = uniform_mdouble(rng, m, M, K), uniform_mdouble(rng, m, K, N)
    else:
        A, B = loguniform_mdouble(rng, m, M, K, lo, -lo), loguniform_mdouble(rng, m, K, N, lo, -lo)
    plan = mw.mw_plan_gemm(m, "textbook", M, N, K, 0, 0)
    C = mw.mw_gemm(to_dev(A, cuda), to_dev(B, cuda), plan).cpu().numpy()
    ref = textbook.TextbookC().gemm(A, B)
    assert np.array_equal(C, ref)
    ratio = exact.exact_product_full(A, B).error_ratio(C).max()
    record_worst(f"textbook m={m} {M}x{N}x{K}", ratio)
    assert ratio <= 1.0


@pytest.mark.parametrize("transA,transB", [(True, False), (False, True), (True, True)])
def test_textbook_transposes(mw, cuda, transA, transB):
    rng = SplitMix64(1310)
    m, M, N, K = 4, 21, 30, 40
    A = uniform_mdouble(rng, m, K, M) if transA else uniform_mdouble(rng, m, M, K)
    B = uniform_mdouble(rng, m, N, K) if transB else uniform_mdouble(rng, m, K, N)
    plan = mw.mw_plan_gemm(m, "textbook", M, N, K, 0, 0)
    C = mw.mw_gemm(to_dev(A, cuda), to_dev(B, cuda), plan, transA=transA, transB=transB)
    ref = textbook.TextbookC().gemm(logical(A, transA), logical(B, transB))
    assert np.array_equal(C.cpu().numpy(), ref)


def test_textbook_rejects_hexa_doubles(mw):
    with pytest.raises(mw.MWError):
        mw.mw_plan_gemm(16, "textbook", 4, 4, 4, 0, 0)
