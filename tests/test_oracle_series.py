"""Pins of the power-series oracle (oracle/series.py): the exact convolution
against polynomial products computed another way and closed forms; the
error-free summation of every coefficient within its bound."""
from fractions import Fraction

import numpy as np

from oracle import exact, series
from synthetic import SplitMix64, uniform_mdouble


def words(vals, m):
    """Exact rationals as m-double series (greedy words), shape (m, n)."""
    return np.array([exact.greedy_words(Fraction(v), m) for v in vals]).T.copy()


def test_exact_convolution_is_the_polynomial_product():
    """Against numpy's convolution of object arrays of Fractions (another route to
    the same polynomial product)."""
    rng = SplitMix64(1100)
    a, b = uniform_mdouble(rng, 2, 1, 9)[:, 0, :], uniform_mdouble(rng, 2, 1, 9)[:, 0, :]
    A = np.array(series.coefficients(a), dtype=object)
    B = np.array(series.coefficients(b), dtype=object)
    want = np.convolve(A, B)[:9]
    assert list(want) == series.convolution_exact(a, b)


def test_closed_forms():
    """(1 - x)(1 + x + x^2 + ...) = 1; a = 1 leaves b unchanged; the square of
    1 + x + x^2 + ... has coefficients i + 1; 1/(1-x)^2 times (1-x) is 1/(1-x)."""
    n, m = 12, 4
    one_minus_x = words([1, -1] + [0] * (n - 2), m)
    geometric = words([1] * n, m)
    unit = words([1] + [0] * (n - 1), m)
    assert series.convolution_exact(one_minus_x, geometric) == [1] + [0] * (n - 1)
    rng = SplitMix64(1101)
    b = uniform_mdouble(rng, m, 1, n)[:, 0, :]
    assert series.convolution_exact(unit, b) == series.coefficients(b)
    assert series.convolution_exact(geometric, geometric) == [i + 1 for i in range(n)]
    square = words([i + 1 for i in range(n)], m)
    assert series.convolution_exact(square, one_minus_x) == [1] * n
    # the sliced form reaches the same exact values (all products of small integers)
    got = series.convolution_sliced(square, one_minus_x, 24, 10, 13)
    assert np.array_equal(got, words([1] * n, m))


def test_sliced_convolution_within_the_bound():
    """A plan that covers the shortest inner product (c_0 = a_0 b_0) meets every
    coefficient's bound; dropping diagonals breaks it."""
    # the short plans drop diagonals whose pairs weigh about 2^-92 (m = 2) and
    # 2^-188 (m = 4) of |a||b|, above 2^(-52m)
    for m, S, D, D_short in ((2, 6, 8, 2), (4, 10, 13, 6)):
        rng = SplitMix64(1110 + m)
        a, b = uniform_mdouble(rng, m, 1, 16)[:, 0, :], uniform_mdouble(rng, m, 1, 16)[:, 0, :]
        got = series.convolution_sliced(a, b, 24, S, D)
        ex = series.convolution_exact(a, b)
        bd = series.convolution_bound(a, b)
        for i in range(16):
            assert abs(exact.to_fraction(got[:, i]) - ex[i]) <= bd[i], i
        short = series.convolution_sliced(a, b, 24, S, D_short)
        assert any(abs(exact.to_fraction(short[:, i]) - ex[i]) > bd[i] for i in range(16))
