"""Error-free summation of split pieces (oracle part O3; test infrastructure only).

Section 2 of the paper assumes the doubles share one exponent, works with the
fraction bits as integers, cuts every double into pieces whose high bits are
zero (quarters of 13 bits for double doubles), sums the products of pieces
exactly in double arithmetic while the number of terms stays below a
threshold, groups them into the diagonal convolutions

    s_i = sum_k sum_{j=0..i} x_{k,j} y_{k,i-j}

and adds s_0 + s_1 + ... at the end ("fuse").  The conclusions (Section 4)
note that these convolutions turn m-double inner products into ordinary matrix
products.  This module states that method for a matrix product C = A B with
the readings the GPU library follows:

* shared exponent per row of A and per column of B (the paper's single shared
  exponent, applied to each inner product separately):
  e(x) = max over the nonzero words x_j of (ilogb(x_j) + 1), so |x_j| < 2^e;
  E_r = max over the row of e (0 for an all-zero row);
* fixed point: with S pieces of w bits, F_r = w S - 2 - E_r and
  T = sum_j trunc(x_j 2^F_r) (every word truncated toward zero on its own, as
  the paper cuts hi and lo words separately), -2^(wS-1) <= T < 2^(wS-1)
  required (the two's complement range of wS bits; the digit bounds below
  hold on it);
* pieces: the balanced base-2^w digits of T, d_0 most significant,
  T = sum_p d_p 2^(w(S-1-p)), -2^(w-1) <= d_p <= 2^(w-1); digit p of row r
  weighs 2^(E_r + 2 - w(p+1));
* diagonal sums s_t = sum_{p+q=t} sum_k dA_{p,ik} dB_{q,kj} for t < D
  (pairs with p < S_A, q < S_B), exact integers;
* fusion: X_ij = sum_t s_t 2^(w(D-1-t)), value X_ij 2^(E_i+E_j+4-w(D+1)),
  rounded greedily into m nonoverlapping doubles.

Everything is exact integer arithmetic (Python ints, numpy int64 products
checked against overflow) and follows the steps in the paper's order.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import Sequence

import numpy as np

from .exact import double_parts, greedy_words


def ilogb(x: float) -> int:
    """floor(log2 |x|) for a nonzero double.
    Section 2: the exponent a shared grid is built on."""
    return math.frexp(x)[1] - 1


def entry_exponent(words: Sequence[float]) -> int | None:
    """max over nonzero words of ilogb + 1, None when every word is zero.
    Section 2: the shared-exponent assumption, taken per row (column) over all words."""
    es = [ilogb(float(x)) + 1 for x in words if x != 0.0]
    return max(es) if es else None


def logical(X: np.ndarray, trans: bool) -> np.ndarray:
    """Operand as (m, R, K): R the output dimension, K the reduction.
    A (not transposed) is already (m, M, K); B (K x N) is used as B^T.
    Transposes as BLAS 'N'/'T' (no passage: the paper has no API)."""
    return np.ascontiguousarray(X.transpose(0, 2, 1)) if trans else X


def row_exponents(L: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(E_r, range_r) for every row of a logical operand L (m, R, K).
    range_r = E_r - min over nonzero entries of e (0 for an all-zero row).
    Section 2: one shared exponent per row of op(A) (column of op(B)) and the spread from it."""
    m, R, K = L.shape
    E = np.zeros(R, dtype=np.int64)
    rng = np.zeros(R, dtype=np.int64)
    for r in range(R):
        es = [entry_exponent(L[:, r, k]) for k in range(K)]
        es = [e for e in es if e is not None]
        if es:
            E[r] = max(es)
            rng[r] = max(es) - min(es)
    return E, rng


def fixed_point(words: Sequence[float], F: int) -> int:
    """sum_j trunc(x_j 2^F), each word truncated toward zero.
    Section 2: every word on the shared fixed-point grid, truncated toward zero."""
    T = 0
    for x in words:
        M, e = double_parts(float(x))
        if M == 0:
            continue
        sh = e + F
        if sh >= 0:
            T += M << sh
        else:
            mag = abs(M) >> (-sh)
            T += mag if M > 0 else -mag
    return T


def balanced_digits(T: int, w: int, S: int) -> list[int]:
    """Digits d_0..d_{S-1} (d_0 most significant) of T in balanced base 2^w:
    the low S-1 digits lie in [-2^(w-1), 2^(w-1)), d_0 takes what is left.
    Section 2 (Figure 1): the cut into pieces whose high bits are zero, as balanced digits."""
    half, base = 1 << (w - 1), 1 << w
    digits = [0] * S
    r = T
    for p in range(S - 1, 0, -1):
        d = ((r + half) % base) - half
        digits[p] = d
        r = (r - d) >> w            # exact: r - d is a multiple of 2^w
    digits[0] = r
    return digits


def bitfield_digits(T: int, w: int, S: int) -> list[int]:
    """Plain w-bit fields of |T| carrying T's sign (the paper's quarters).
    Section 2 (Figure 1)."""
    sgn = -1 if T < 0 else 1
    a = abs(T)
    mask = (1 << w) - 1
    return [sgn * ((a >> (w * (S - 1 - p))) & mask) for p in range(S)]


class Split:
    """Digits of a logical operand L (m, R, K): ``digits[p, r, k]``, ``E[r]``.
    Section 2: steps 1 and 2 (shared exponent, pieces) for one operand."""

    def __init__(self, L: np.ndarray, w: int, S: int, rows: Sequence[int] | None = None):
        m, R, K = L.shape
        self.w, self.S = w, S
        self.rows = list(range(R)) if rows is None else list(rows)
        E_all, rng_all = row_exponents(L[:, self.rows, :])
        self.E = E_all
        self.range = rng_all
        self.digits = np.zeros((S, len(self.rows), K), dtype=np.int64)
        self.T = [[0] * K for _ in self.rows]
        self.in_range = True
        lim = 1 << (w * S - 1)
        for a, r in enumerate(self.rows):
            F = w * S - 2 - int(self.E[a])
            for k in range(K):
                T = fixed_point(L[:, r, k], F)
                self.T[a][k] = T
                if not (-lim <= T < lim):
                    self.in_range = False
                d = balanced_digits(T, w, S)
                for p in range(S):
                    self.digits[p, a, k] = d[p]

    def digit_weight_exponent(self, a: int, p: int) -> int:
        """Digit p of (local) row a weighs 2^(E + 2 - w(p+1)).
        Section 2: the weight of a piece on the shared grid."""
        return int(self.E[a]) + 2 - self.w * (p + 1)


def pairs(S_A: int, S_B: int, D: int) -> list[tuple[int, int]]:
    """Kept (p, q): p < S_A, q < S_B, p + q < D, ordered by diagonal then p.
    Section 2: the products of pieces kept, by diagonal p + q."""
    return [(p, t - p) for t in range(D) for p in range(S_A) if 0 <= t - p < S_B]


def diagonal_sums(dA: np.ndarray, dB: np.ndarray, D: int) -> np.ndarray:
    """s[t, i, j] = sum_{p+q=t} sum_k dA[p, i, k] dB[q, j, k]  (Section 2 s_i).

    Products of digit matrices use numpy's int64 matmul (an exact integer
    library primitive) while the magnitude bound rules out overflow, and
    Python integers (numpy object arrays, exact at any size) otherwise."""
    S_A, M, K = dA.shape
    S_B, N, K2 = dB.shape
    assert K == K2
    amax = int(np.abs(dA).max()) if dA.size else 0
    bmax = int(np.abs(dB).max()) if dB.size else 0
    if amax * bmax * K * min(S_A, S_B) < (1 << 62):
        s = np.zeros((D, M, N), dtype=np.int64)
        for p, q in pairs(S_A, S_B, D):
            s[p + q] += dA[p] @ dB[q].T
        return s
    oA, oB = dA.astype(object), dB.astype(object)
    s = np.zeros((D, M, N), dtype=object)
    for p, q in pairs(S_A, S_B, D):
        s[p + q] = s[p + q] + oA[p].dot(oB[q].T)
    return s


def fuse_integer(s_ij: Sequence[int], w: int, D: int) -> int:
    """X = sum_t s_t 2^(w(D-1-t)).
    Section 2: the diagonal sums s_i scaled by their weights; Section 4: added once at the end."""
    X = 0
    for t in range(D):
        X += int(s_ij[t]) << (w * (D - 1 - t))
    return X


def fused_value(s_ij: Sequence[int], w: int, D: int, EA: int, EB: int) -> Fraction:
    """Section 2 and Section 4: the fused exact value with the shared exponents applied."""
    X = fuse_integer(s_ij, w, D)
    return Fraction(X) * Fraction(2) ** (EA + EB + 4 - w * (D + 1))


def group_values(s_ij: Sequence[int], w: int, bounds: Sequence[tuple[int, int]]) -> list[int]:
    """V_g = sum_{t=t0..t1} s_t 2^(w(t1 - t)) for each group [t0, t1] of diagonals.
    Section 2's diagonal sums joined in groups by Horner's rule (equal to fuse_integer on each group)."""
    out = []
    for t0, t1 in bounds:
        V = 0
        for t in range(t0, t1 + 1):
            V += int(s_ij[t]) << (w * (t1 - t))
        out.append(V)
    return out


class SlicedProduct:
    """The whole method on a block of outputs: split A's rows and B's columns,
    diagonal sums, exact fusion, greedy rounding to m words.
    Sections 2 and 4: the whole error-free summation on a block of outputs."""

    def __init__(self, A: np.ndarray, B: np.ndarray, w: int, S_A: int, S_B: int, D: int,
                 rows: Sequence[int] | None = None, cols: Sequence[int] | None = None,
                 transA: bool = False, transB: bool = False):
        LA = logical(A, transA)                      # (m, M, K)
        LB = logical(B, not transB)                  # (m, N, K)
        self.m = LA.shape[0]
        self.w, self.S_A, self.S_B, self.D = w, S_A, S_B, D
        self.A = Split(LA, w, S_A, rows)
        self.B = Split(LB, w, S_B, cols)
        self.s = diagonal_sums(self.A.digits, self.B.digits, D)

    def value(self, a: int, b: int) -> Fraction:
        """Sections 2 and 4: the fused exact value of one output."""
        return fused_value(self.s[:, a, b], self.w, self.D, int(self.A.E[a]), int(self.B.E[b]))

    def words(self, a: int, b: int) -> list[float]:
        """Sections 2 and 4: the m words of one output."""
        return greedy_words(self.value(a, b), self.m)

    def result(self) -> np.ndarray:
        """Greedy-rounded m words for the selected block, shape (m, rows, cols).
        Sections 2 and 4."""
        R, C = len(self.A.rows), len(self.B.rows)
        out = np.zeros((self.m, R, C))
        for a in range(R):
            for b in range(C):
                out[:, a, b] = self.words(a, b)
        return out
