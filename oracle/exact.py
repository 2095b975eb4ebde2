"""Exact arithmetic on m-doubles (oracle part O2; test infrastructure only).

An m-double is an unevaluated sum of doubles x_0 + ... + x_{m-1} (Section 1).
Every double is a dyadic rational M 2^e with an integer M of at most 53 bits,
so every value here is held exactly as a Python integer times a power of two;
no floating-point operation touches a value before the final rounding.

Definitions used by the tests:

* exact product   C_ij = sum_k a_ik b_kj over the exact values of the entries;
* error bound     bound_ij = 2 K 2^(-52 m) sum_k |a_ik| |b_kj|  (the accuracy
                  the product must reach, componentwise);
* greedy rounding c_0 = RN(v), c_1 = RN(v - c_0), ...: the m nonoverlapping
                  doubles of an exact value v (RN = round to nearest even).

Matrices are numpy arrays of shape (m, rows, cols), plane j holding word j.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import Iterable, Sequence

import numpy as np


def double_parts(x: float) -> tuple[int, int]:
    """(M, e) with x == M * 2**e exactly, M an integer (0, 0 for zero).
    Section 1: a word of an m-double is an ordinary double."""
    if x == 0.0:
        return 0, 0
    if not math.isfinite(x):
        raise ValueError("non-finite double")
    mant, ex = math.frexp(x)          # x = mant * 2**ex, 0.5 <= |mant| < 1
    return int(mant * (1 << 53)), ex - 53


def min_exponent(X: np.ndarray) -> int:
    """Smallest e over the nonzero words of X (scale that makes all words integers).
    Section 1: the value of an m-double is the exact sum of its words."""
    nz = X[X != 0.0]
    if nz.size == 0:
        return 0
    _, ex = np.frexp(nz)
    return int(ex.min()) - 53


def entry_int(words: Iterable[float], scale: int) -> int:
    """Exact value of an m-double times 2**(-scale), as an integer.
    ``scale`` must not exceed the exponent of any nonzero word.
    Section 1: the value of an m-double is the exact sum of its words."""
    total = 0
    for x in words:
        M, e = double_parts(float(x))
        if M == 0:
            continue
        sh = e - scale
        if sh < 0:
            raise ValueError("scale above a word's exponent")
        total += M << sh
    return total


def to_fraction(words: Iterable[float]) -> Fraction:
    """Exact value of an m-double (Section 1: the unevaluated sum of its words)."""
    total = Fraction(0)
    for x in words:
        total += Fraction(float(x))
    return total


def exact_rows(X: np.ndarray, rows: Sequence[int], scale: int) -> list[list[int]]:
    """Exact integer values (times 2**-scale) of the listed rows of X.
    Section 1: exact values of the entries."""
    m = X.shape[0]
    return [[entry_int((X[j, r, c] for j in range(m)), scale) for c in range(X.shape[2])]
            for r in rows]


def exact_cols(X: np.ndarray, cols: Sequence[int], scale: int) -> list[list[int]]:
    """Exact integer values (times 2**-scale) of the listed columns of X,
    returned as one list per column (index k along the rows of X).
    Section 1: exact values of the entries."""
    m = X.shape[0]
    return [[entry_int((X[j, r, c] for j in range(m)), scale) for r in range(X.shape[1])]
            for c in cols]


class ExactProduct:
    """Exact C = A B (and sum_k |a_ik||b_kj|) on a chosen block of outputs.

    A has shape (m, M, K) and B (m, K, N).  ``rows`` and ``cols`` select the
    outputs; each needs only its own row of A and column of B.
    The exact matrix product the method approximates (Section 4's matrix form)."""

    def __init__(self, A: np.ndarray, B: np.ndarray, rows: Sequence[int], cols: Sequence[int]):
        assert A.shape[0] == B.shape[0] and A.shape[2] == B.shape[1]
        self.m = A.shape[0]
        self.K = A.shape[2]
        self.rows, self.cols = list(rows), list(cols)
        self.sa = min_exponent(A[:, self.rows, :])
        self.sb = min_exponent(B[:, :, self.cols])
        self.scale = self.sa + self.sb           # value = integer * 2**scale
        ar = exact_rows(A, self.rows, self.sa)
        bc = exact_cols(B, self.cols, self.sb)
        self.value = [[sum(x * y for x, y in zip(a, b)) for b in bc] for a in ar]
        self.absum = [[sum(abs(x) * abs(y) for x, y in zip(a, b)) for b in bc] for a in ar]

    def exact(self, r: int, c: int) -> Fraction:
        """Exact C for local output (r, c) (Section 4's matrix form)."""
        return Fraction(self.value[r][c]) * Fraction(2) ** self.scale

    def bound(self, r: int, c: int) -> Fraction:
        """2 K 2^(-52 m) sum_k |a_rk||b_kc| for output (rows[r], cols[c]).
        The componentwise bound the library targets (the paper sums exactly and states no matrix bound)."""
        return (Fraction(2 * self.K) * Fraction(self.absum[r][c])
                * Fraction(2) ** (self.scale - 52 * self.m))

    def error_ratio(self, C: np.ndarray) -> np.ndarray:
        """|C - C_exact| / bound for every selected output, C of shape (m, M, N)
        (the full product; only the selected outputs are read).  Returns a float
        array (rows x cols); inf where the bound is 0 but the error is not.
        Against the componentwise bound (see bound)."""
        out = np.zeros((len(self.rows), len(self.cols)))
        for a, r in enumerate(self.rows):
            for b, c in enumerate(self.cols):
                err = abs(to_fraction(C[:, r, c]) - self.exact(a, b))
                bnd = self.bound(a, b)
                if err == 0:
                    out[a, b] = 0.0
                elif bnd == 0:
                    out[a, b] = math.inf
                else:
                    out[a, b] = float(err / bnd)
        return out


def exact_product_full(A: np.ndarray, B: np.ndarray) -> ExactProduct:
    """ExactProduct over every output (Section 4's matrix form)."""
    return ExactProduct(A, B, range(A.shape[1]), range(B.shape[2]))


def round_nearest(v: Fraction) -> float:
    """RN(v), ties to even: Python's int/int true division rounds correctly.
    Section 2: the final step rounds the exact sum into doubles."""
    return v.numerator / v.denominator if v != 0 else 0.0


def greedy_words(v: Fraction, m: int) -> list[float]:
    """c_0 = RN(v), c_j = RN(v - c_0 - ... - c_{j-1}): nonoverlapping words.
    Section 2 and Section 4: the exact sum, renormalised once at the end into m nonoverlapping words (greedy reading)."""
    words = []
    r = v
    for _ in range(m):
        c = round_nearest(r)
        words.append(c)
        r -= Fraction(c)
    return words


def nonoverlapping(words: Sequence[float]) -> bool:
    """|x_{j+1}| <= ulp(x_j) for consecutive nonzero words, zeros only at the tail.
    Section 1: the words of an m-double do not overlap."""
    seen_zero = False
    for a, b in zip(words[:-1], words[1:]):
        if a == 0.0:
            seen_zero = True
        if seen_zero and b != 0.0:
            return False
        if a != 0.0 and abs(b) > math.ulp(a):
            return False
    return True
