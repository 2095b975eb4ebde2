"""Products of truncated power series with m-double coefficients (oracle;
test infrastructure only).

Section 1 of the paper motivates multiword arithmetic with power series, and
Section 2's diagonal sums s_i are convolutions: the coefficient of x^i in the
product of a(x) = sum_k a_k x^k and b(x) = sum_k b_k x^k is

    c_i = sum_{k=0..i} a_k b_{i-k},

an inner product of a_0..a_i with b_i..b_0.  The product of two series
truncated to n coefficients keeps c_0..c_{n-1}.

* ``convolution_exact``  -- every c_i as an exact rational (Fractions of the
  m-doubles' exact values): the definition.
* ``convolution_bound``  -- 2 (i+1) 2^(-52m) sum_k |a_k||b_{i-k}|, the
  componentwise bound the library meets for each coefficient (the inner
  product's bound with K = i+1).
* ``convolution_sliced`` -- the error-free summation of Section 2 applied to
  each coefficient's inner product with the given plan (w, S, D), through
  ``slicing.SlicedProduct``: the words the library's kernel must produce bit
  for bit.

Series are numpy arrays of shape (m, n): word j of coefficient k at [j, k].
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from .exact import to_fraction
from .slicing import SlicedProduct


def coefficients(a: np.ndarray) -> list[Fraction]:
    """Exact value of every coefficient (Section 1: an m-double is the sum of its words)."""
    return [to_fraction(a[:, k]) for k in range(a.shape[1])]


def convolution_exact(a: np.ndarray, b: np.ndarray) -> list[Fraction]:
    """c_i = sum_{k <= i} a_k b_{i-k} for i < n, exactly."""
    A, B = coefficients(a), coefficients(b)
    n = len(A)
    return [sum((A[k] * B[i - k] for k in range(i + 1)), Fraction(0)) for i in range(n)]


def convolution_bound(a: np.ndarray, b: np.ndarray) -> list[Fraction]:
    """2 (i+1) 2^(-52m) sum_{k <= i} |a_k| |b_{i-k}| for every coefficient."""
    m = a.shape[0]
    A, B = coefficients(a), coefficients(b)
    n = len(A)
    return [Fraction(2 * (i + 1)) * Fraction(2) ** (-52 * m)
            * sum((abs(A[k]) * abs(B[i - k]) for k in range(i + 1)), Fraction(0))
            for i in range(n)]


def convolution_sliced(a: np.ndarray, b: np.ndarray, w: int, S: int, D: int) -> np.ndarray:
    """The m words of every c_i by the error-free summation with the plan (w, S, D):
    the inner product of a_0..a_i (a 1 x (i+1) row) with b_i..b_0 (a column)."""
    m, n = a.shape
    out = np.zeros((m, n))
    for i in range(n):
        row = np.ascontiguousarray(a[:, None, :i + 1])                  # (m, 1, i+1)
        col = np.ascontiguousarray(b[:, i::-1][:, :, None])             # (m, i+1, 1)
        out[:, i] = SlicedProduct(row, col, w, S, S, D).result()[:, 0, 0]
    return out
