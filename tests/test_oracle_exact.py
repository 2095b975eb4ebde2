"""Pins for the exact part of the oracle (O2): values, exact product, bound,
greedy rounding.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact
from synthetic import SplitMix64, paper_pattern_mdouble, uniform_mdouble, loguniform_mdouble


def brute_product(A, B):
    """C = A B with fractions.Fraction, entry by entry (tiny sizes only)."""
    m, M, K = A.shape
    N = B.shape[2]
    out = [[Fraction(0)] * N for _ in range(M)]
    for i in range(M):
        for j in range(N):
            s = Fraction(0)
            for k in range(K):
                a = sum(Fraction(float(A[w, i, k])) for w in range(m))
                b = sum(Fraction(float(B[w, k, j])) for w in range(m))
                s += a * b
            out[i][j] = s
    return out


def test_double_parts_roundtrip():
    rng = SplitMix64(5)
    xs = list(rng.sym(200)) + [1.0, -1.0, 2.0 ** -1074, -(2.0 ** 1023), 0.5, 3.0]
    for x in xs:
        M, e = exact.double_parts(float(x))
        assert Fraction(M) * Fraction(2) ** e == Fraction(float(x))
        assert abs(M) < 2 ** 53


@pytest.mark.parametrize("gen", ["uniform", "loguniform", "pattern"])
@pytest.mark.parametrize("m", [2, 4])
def test_exact_product_matches_fractions(gen, m):
    rng = SplitMix64(100 + m)
    if gen == "uniform":
        A, B = uniform_mdouble(rng, m, 5, 7), uniform_mdouble(rng, m, 7, 4)
    elif gen == "loguniform":
        A, B = loguniform_mdouble(rng, m, 5, 7, -20, 20), loguniform_mdouble(rng, m, 7, 4, -20, 20)
    else:
        A, B = paper_pattern_mdouble(rng, m, 5, 7), paper_pattern_mdouble(rng, m, 7, 4)
    ex = exact.exact_product_full(A, B)
    ref = brute_product(A, B)
    for i in range(5):
        for j in range(4):
            assert ex.exact(i, j) == ref[i][j]


def test_m1_reduces_to_integer_gemm():
    """With one word per entry and small integer entries the product is the
    integer matrix product (numpy int64 matmul)."""
    rng = SplitMix64(9)
    Ai = (rng.next(6 * 9) % np.uint64(2001)).astype(np.int64).reshape(6, 9) - 1000
    Bi = (rng.next(9 * 5) % np.uint64(2001)).astype(np.int64).reshape(9, 5) - 1000
    ex = exact.exact_product_full(Ai[None].astype(np.float64), Bi[None].astype(np.float64))
    C = Ai @ Bi
    for i in range(6):
        for j in range(5):
            assert ex.exact(i, j) == C[i, j]


def test_identity_gives_a():
    rng = SplitMix64(10)
    A = uniform_mdouble(rng, 4, 6, 6)
    I = np.zeros((4, 6, 6))
    I[0] = np.eye(6)
    ex = exact.exact_product_full(A, I)
    for i in range(6):
        for j in range(6):
            assert ex.exact(i, j) == exact.to_fraction(A[:, i, j])


def test_bound_formula_on_small_integers():
    """bound = 2K 2^(-52m) sum_k |a||b|: check on integer data where the sum
    is known in closed form."""
    A = np.zeros((2, 1, 3)); A[0] = [[1.0, -2.0, 3.0]]
    B = np.zeros((2, 3, 1)); B[0] = [[4.0], [5.0], [-6.0]]
    ex = exact.exact_product_full(A, B)
    assert ex.exact(0, 0) == 4 - 10 - 18
    assert ex.bound(0, 0) == Fraction(2 * 3 * (4 + 10 + 18)) * Fraction(2) ** (-104)


def test_greedy_words_closed_forms():
    # 1 + 2^-60 + 2^-130 splits into its three powers of two
    v = Fraction(1) + Fraction(2) ** -60 + Fraction(2) ** -130
    assert exact.greedy_words(v, 3) == [1.0, 2.0 ** -60, 2.0 ** -130]
    # 1/3: every word is RN of the remainder, the remainder shrinks by 2^-53 per word
    third = Fraction(1, 3)
    w = exact.greedy_words(third, 4)
    assert w[0] == 1.0 / 3.0
    rem = third - sum(Fraction(x) for x in w)
    assert abs(rem) <= Fraction(2) ** (-2 - 53 * 4)
    assert exact.nonoverlapping(w)
    # ties go to even: 1 + 2^-53 rounds to 1 and leaves 2^-53
    assert exact.greedy_words(Fraction(1) + Fraction(2) ** -53, 2) == [1.0, 2.0 ** -53]


def test_greedy_words_random_accuracy():
    rng = SplitMix64(12)
    X = loguniform_mdouble(rng, 8, 1, 50, -30, 30)
    for k in range(50):
        v = exact.to_fraction(X[:, 0, k]) * Fraction(1, 7)
        for m in (2, 4, 8):
            w = exact.greedy_words(v, m)
            assert exact.nonoverlapping(w)
            assert abs(v - sum(Fraction(x) for x in w)) <= abs(v) * Fraction(2) ** (-53 * m)


def test_error_ratio_detects_a_dropped_word():
    """A planted mistake on the CPU: dropping the last word of a correct result
    must exceed the bound, keeping it must not."""
    rng = SplitMix64(13)
    A, B = uniform_mdouble(rng, 2, 4, 16), uniform_mdouble(rng, 2, 16, 4)
    ex = exact.exact_product_full(A, B)
    C = np.zeros((2, 4, 4))
    for i in range(4):
        for j in range(4):
            C[:, i, j] = exact.greedy_words(ex.exact(i, j), 2)
    assert ex.error_ratio(C).max() < 1.0 / 16
    bad = C.copy()
    bad[1] = 0.0
    assert ex.error_ratio(bad).max() > 1.0
