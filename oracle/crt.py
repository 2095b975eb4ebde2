"""Products of fixed-point integers through residues (oracle part O4; test
infrastructure only).

Section 4 of the paper points at the Ozaki scheme as the way to bring the
error-free summation onto tensor cores, and Section 1 calls the split into
pieces a stepping stone towards it.  Its second scheme (the "Ozaki scheme II"
of Ozaki, Uchino and Imamura) replaces the products of pieces by products of
residues: instead of cutting the fixed-point integers into w-bit digits and
multiplying every pair of digit matrices, it reduces them modulo a few small
pairwise coprime moduli, multiplies one residue matrix per modulus, and
recovers the exact integer products with the Chinese remainder theorem.  This
module states that computation for C = A B with the readings the GPU library
follows:

* shared exponents and fixed point exactly as in ``slicing`` (one exponent
  per row of A and per column of B, every word truncated toward zero on its
  own): with L_A fixed-point bits, T^A_ik = sum_j trunc(a_ik,j 2^(L_A-2-E_i)),
  -2^(L_A-1) <= T^A_ik < 2^(L_A-1); the same for B with L_B (this is
  ``slicing.Split``'s T with w = 1 and S = L);
* the exact integer product X_ij = sum_k T^A_ik T^B_jk, whose value
  X_ij 2^(E_i+E_j+4-L_A-L_B) is rounded greedily into m words;
* moduli p_1..p_n, pairwise coprime, P = p_1 ... p_n; balanced residues
  r = T mod p in [-floor(p/2), ceil(p/2) - 1];
* per modulus the exact integer sums Y_i = sum_k r^A_i,ik r^B_i,jk (what one
  tensor-core product of residue matrices computes);
* reconstruction: X is the unique integer in (-P/2, P/2] with X = Y_i mod p_i
  for every i, which equals the exact product whenever |X| < P/2.

Everything is exact integer arithmetic (Python ints; numpy int64 products only
where the magnitude bound rules out overflow).  The moduli are an input: any
pairwise coprime set whose product is large enough gives the same X.
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import Sequence

import numpy as np

from .exact import greedy_words
from .slicing import fixed_point, logical, row_exponents


def pairwise_coprime(moduli: Sequence[int]) -> bool:
    """Every two moduli share no factor (the Chinese remainder theorem's hypothesis)."""
    ms = [int(p) for p in moduli]
    return all(p >= 2 for p in ms) and all(
        math.gcd(ms[i], ms[j]) == 1 for i in range(len(ms)) for j in range(i + 1, len(ms)))


def modulus_product(moduli: Sequence[int]) -> int:
    """P = p_1 ... p_n."""
    P = 1
    for p in moduli:
        P *= int(p)
    return P


def balanced_residue(x: int, p: int) -> int:
    """The residue of x modulo p in [-floor(p/2), ceil(p/2) - 1] (at most
    floor(p/2) in magnitude, so p <= 513 keeps it within bfloat16's exact
    integers)."""
    h = p // 2
    return ((int(x) + h) % p) - h


def crt_reconstruct(ys: Sequence[int], moduli: Sequence[int]) -> int:
    """The unique X in (-P/2, P/2] with X = ys[i] mod moduli[i] for every i
    (Chinese remainder theorem, written out with the inverses of P/p_i)."""
    P = modulus_product(moduli)
    X = 0
    for y, p in zip(ys, moduli):
        Q = P // p
        X += (int(y) % p) * Q * pow(Q % p, -1, p)
    X %= P
    return X - P if 2 * X > P else X


class ResidueSplit:
    """Fixed-point integers T (rows x K) and their balanced residues of a
    logical operand L (m, R, K) with L_bits fixed-point bits per entry."""

    def __init__(self, L: np.ndarray, L_bits: int, moduli: Sequence[int],
                 rows: Sequence[int] | None = None):
        m, R, K = L.shape
        self.L_bits = L_bits
        self.rows = list(range(R)) if rows is None else list(rows)
        self.E, self.range = row_exponents(L[:, self.rows, :])
        lim = 1 << (L_bits - 1)
        self.in_range = True
        self.T = []
        for a, r in enumerate(self.rows):
            F = L_bits - 2 - int(self.E[a])
            row = [fixed_point(L[:, r, k], F) for k in range(K)]
            self.in_range &= all(-lim <= t < lim for t in row)
            self.T.append(row)
        # balanced_residue of every T, over an object array of Python integers
        Tobj = np.array(self.T, dtype=object).reshape(len(self.rows), K)
        self.residues = np.zeros((len(moduli), len(self.rows), K), dtype=np.int64)
        for i, p in enumerate(moduli):
            h = int(p) // 2
            self.residues[i] = (((Tobj + h) % int(p)) - h).astype(np.int64)


def residue_products(RA: np.ndarray, RB: np.ndarray) -> np.ndarray:
    """Y[i, a, b] = sum_k RA[i, a, k] RB[i, b, k]: one integer matrix product
    per modulus, exact (|r| <= 256 and K < 2^46 keep int64 far from overflow)."""
    n, Ma, K = RA.shape
    assert RB.shape[0] == n and RB.shape[2] == K
    amax = int(np.abs(RA).max()) if RA.size else 0
    bmax = int(np.abs(RB).max()) if RB.size else 0
    assert amax * bmax * K < (1 << 62)
    return np.stack([RA[i] @ RB[i].T for i in range(n)]) if n else np.zeros((0, Ma, RB.shape[1]),
                                                                           dtype=np.int64)


class ResidueProduct:
    """The whole residue form on a block of outputs: fixed-point split of A's
    rows and B's columns, residue products per modulus, reconstruction by the
    Chinese remainder theorem, greedy rounding to m words."""

    def __init__(self, A: np.ndarray, B: np.ndarray, L_A: int, L_B: int,
                 moduli: Sequence[int], rows: Sequence[int] | None = None,
                 cols: Sequence[int] | None = None, transA: bool = False,
                 transB: bool = False):
        assert pairwise_coprime(moduli)
        LA = logical(A, transA)                      # (m, M, K)
        LB = logical(B, not transB)                  # (m, N, K)
        self.m = LA.shape[0]
        self.K = LA.shape[2]
        self.L_A, self.L_B = L_A, L_B
        self.moduli = [int(p) for p in moduli]
        self.A = ResidueSplit(LA, L_A, self.moduli, rows)
        self.B = ResidueSplit(LB, L_B, self.moduli, cols)
        self.Y = residue_products(self.A.residues, self.B.residues)

    def X(self, a: int, b: int) -> int:
        """The reconstructed integer of local output (a, b)."""
        return crt_reconstruct([int(y) for y in self.Y[:, a, b]], self.moduli)

    def X_direct(self, a: int, b: int) -> int:
        """sum_k T^A_ak T^B_bk computed directly (no residues), for the pins."""
        return sum(x * y for x, y in zip(self.A.T[a], self.B.T[b]))

    def value(self, a: int, b: int) -> Fraction:
        """The exact value X 2^(E_a + E_b + 4 - L_A - L_B)."""
        return Fraction(self.X(a, b)) * Fraction(2) ** (
            int(self.A.E[a]) + int(self.B.E[b]) + 4 - self.L_A - self.L_B)

    def words(self, a: int, b: int) -> list[float]:
        return greedy_words(self.value(a, b), self.m)

    def result(self) -> np.ndarray:
        """Greedy-rounded m words for the selected block, shape (m, rows, cols)."""
        R, C = len(self.A.rows), len(self.B.rows)
        out = np.zeros((self.m, R, C))
        for a in range(R):
            for b in range(C):
                out[:, a, b] = self.words(a, b)
        return out


def fixed_point_bits(m: int, K: int, spread: int) -> int:
    """Fixed-point bits per entry for the componentwise bound 2K 2^(-52m) (|A||B|):
    the truncation of one operand costs at most m 2^(spread + 3 - L) of |a||b|
    per term, given a quarter of the budget (the same share as the slice form;
    the residue form drops no products, so that quarter is spare)."""
    return max(2, math.ceil(52 * m + spread + math.log2(m) + 5 - math.log2(K) - 1e-9))


def product_bits_needed(L_A: int, L_B: int, K: int) -> float:
    """log2 of the modulus product P needed: |X| <= K 2^(L_A + L_B - 2) must
    stay below P/8 (P/2 for uniqueness, a factor 4 to spare for the library's
    floating-point estimate of the multiple of P it subtracts)."""
    return L_A + L_B + 1 + math.log2(K)
