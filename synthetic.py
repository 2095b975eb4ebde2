"""Seeded synthetic m-double matrices (input generators only).

This module is shared by the CPU oracle, the GPU tests and the benchmark. It
holds no arithmetic of the m-double product: it only draws random numbers and
shapes them into m structure-of-arrays double planes, shape ``(m, rows, cols)``,
plane 0 holding the leading word of every entry.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state advances by the golden
gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
variant-13 finaliser.  Output i of a stream seeded with s is therefore
``mix(s + (i + 1) * gamma)``, which numpy evaluates for a whole block at once.
A double in [0, 1) takes the top 53 bits of an output; U[-1, 1] is 2u - 1.

Workloads (the paper's application is power series, Section 1; its timing data
pattern is Section 2):

* ``uniform_mdouble``: leading word U[-1, 1]; each lower word is the word
  above times 2^-53 * u with a fresh u ~ U[-1, 1] (double-double inputs of the
  n = 64 exactness case, the batched octo-double products, the adjoint case).
* ``loguniform_mdouble``: leading word 2^U[lo, hi] with a random sign, lower
  words as above (quad-double 1024^3 case: [-8, 8]; 4096^3 Ozaki case:
  [-20, 20]).
* ``paper_pattern_mdouble``: every word a positive double whose 52 fraction
  bits follow the Section 2 pattern ``1 b^12`` four times, the words of one
  entry placed 52 bits apart as in the paper's double doubles (Table 2's
  1,024 inner products of length 6,144: ``table2_operands``).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Counter form of SplitMix64; ``next(n)`` returns the next n outputs."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + idx * GAMMA
            self.state = self.state + np.uint64(n) * GAMMA
            return _mix(z)

    def unit(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) from the top 53 bits."""
        return (self.next(n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53

    def sym(self, n: int) -> np.ndarray:
        """n doubles in [-1, 1)."""
        return 2.0 * self.unit(n) - 1.0

    def bits(self, n: int) -> np.ndarray:
        return self.next(n)


def _lower_words(rng: SplitMix64, lead: np.ndarray, m: int) -> np.ndarray:
    out = np.empty((m,) + lead.shape, dtype=np.float64)
    out[0] = lead
    for j in range(1, m):
        u = rng.sym(lead.size).reshape(lead.shape)
        out[j] = out[j - 1] * 2.0 ** -53 * u
    return out


def uniform_mdouble(rng: SplitMix64, m: int, rows: int, cols: int) -> np.ndarray:
    """Leading word U[-1, 1); lower word j = word j-1 * 2^-53 * U[-1, 1)."""
    lead = rng.sym(rows * cols).reshape(rows, cols)
    return _lower_words(rng, lead, m)


def loguniform_mdouble(rng: SplitMix64, m: int, rows: int, cols: int,
                       lo: float, hi: float) -> np.ndarray:
    """|leading word| = 2^U[lo, hi), random sign; lower words as above."""
    e = lo + (hi - lo) * rng.unit(rows * cols)
    sgn = np.where((rng.bits(rows * cols) >> np.uint64(63)) == 0, 1.0, -1.0)
    lead = (sgn * np.exp2(e)).reshape(rows, cols)
    return _lower_words(rng, lead, m)


def paper_pattern_double(rng: SplitMix64, n: int, exponent: int = 0) -> np.ndarray:
    """n positive doubles 2^exponent * 1.f whose 52-bit fraction f reads
    ``1 b^12`` four times (Section 2 data pattern)."""
    b = rng.bits(n)
    frac = np.zeros(n, dtype=np.uint64)
    for q in range(4):
        twelve = (b >> np.uint64(12 * q)) & np.uint64(0xFFF)
        quarter = np.uint64(1 << 12) | twelve
        frac |= quarter << np.uint64(13 * (3 - q))
    bits = (np.uint64(1023 + exponent) << np.uint64(52)) | frac
    return bits.view(np.float64)


def paper_pattern_mdouble(rng: SplitMix64, m: int, rows: int, cols: int) -> np.ndarray:
    """m-double entries whose every word follows the Section 2 pattern; word j
    has exponent -53 j so the words are nonoverlapping and its 53 significand
    bits continue the bits of word j-1."""
    out = np.empty((m, rows, cols), dtype=np.float64)
    for j in range(m):
        out[j] = paper_pattern_double(rng, rows * cols, exponent=-53 * j).reshape(rows, cols)
    return out


# --- the named workloads -------------------------------------------------------------------

def dd_n64(seed: int = 0, n: int = 64):
    """Double-double A, B (n x n), leading words U[-1,1), seed 0."""
    rng = SplitMix64(seed)
    return uniform_mdouble(rng, 2, n, n), uniform_mdouble(rng, 2, n, n)


def loguniform_pair(m: int, M: int, N: int, K: int, lo: float, hi: float, seed: int):
    """A (M x K) and B (K x N), every leading word 2^U[lo,hi) with a random sign."""
    rng = SplitMix64(seed)
    return (loguniform_mdouble(rng, m, M, K, lo, hi),
            loguniform_mdouble(rng, m, K, N, lo, hi))


def qd_1024(seed: int = 1, n: int = 1024):
    """Quad-double A, B (n x n), magnitudes 2^U[-8, 8), seed 1."""
    return loguniform_pair(4, n, n, n, -8.0, 8.0, seed)


def ozaki_4096(m: int, seed: int = 2, n: int = 4096):
    """m-double A, B (n x n), magnitudes 2^U[-20, 20), seed 2."""
    return loguniform_pair(m, n, n, n, -20.0, 20.0, seed)


def batch_sizes(count: int = 20000, lo: int = 8, hi: int = 128, seed: int = 3) -> np.ndarray:
    """Problem sizes n ~ U{lo..hi} for the batched octo-double products."""
    rng = SplitMix64(seed)
    return (lo + (rng.next(count) % np.uint64(hi - lo + 1))).astype(np.int64)


def batch_problems(sizes: np.ndarray, m: int = 8, seed: int = 3):
    """For each size n, a square pair (A, B) of m-doubles with U[-1,1) leading words.
    The stream continues after the sizes were drawn with the same seed."""
    rng = SplitMix64(seed)
    rng.next(len(sizes))
    out = []
    for n in sizes:
        n = int(n)
        out.append((uniform_mdouble(rng, m, n, n), uniform_mdouble(rng, m, n, n)))
    return out


def batch_flat(sizes: np.ndarray, m: int = 8, seed: int = 3):
    """All square problems of a batch in two flat buffers (every A_i, then every
    B_i, each m planes of n_i x n_i), plus each problem's element offset.
    Leading words U[-1,1), lower words x 2^-53 U[-1,1).  The stream continues
    after the sizes were drawn with the same seed."""
    rng = SplitMix64(seed)
    rng.next(len(sizes))
    n2 = sizes.astype(np.int64) ** 2
    offs = np.concatenate([[0], np.cumsum(n2)[:-1]])
    total = int(n2.sum())
    flats = []
    for _ in range(2):
        lead = rng.sym(total)
        words = _lower_words(rng, lead, m)          # (m, total)
        flats.append(words)
    return flats[0], flats[1], offs


def adjoint_case(seed: int = 4, M: int = 2048, K: int = 1024, N: int = 2048):
    """Double-double A (M x K), B (K x N), and loss weights W (M x N) U[-1,1)."""
    rng = SplitMix64(seed)
    A = uniform_mdouble(rng, 2, M, K)
    B = uniform_mdouble(rng, 2, K, N)
    W = rng.sym(M * N).reshape(M, N)
    return A, B, W


def table2_operands(m: int, count: int = 1024, K: int = 6144, seed: int = 5):
    """Table 2's workload: count inner products of length K, both vectors of
    every product m-doubles on the Section 2 bit pattern; rows of A and B."""
    rng = SplitMix64(seed)
    return paper_pattern_mdouble(rng, m, count, K), paper_pattern_mdouble(rng, m, count, K)
