"""Pins for the error-free summation oracle (O3).  CPU only.

Each check ties the oracle to something outside itself: exact reconstruction,
brute force on tiny inputs, the exact product of ``oracle.exact`` (built from
mantissas, not from digits), closed forms, and the paper's Section 2 pattern.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact, slicing
from synthetic import (SplitMix64, dd_n64, loguniform_mdouble, paper_pattern_double,
                       paper_pattern_mdouble, uniform_mdouble)

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def read_golden(name):
    rows = []
    with open(f"{GOLDEN}/{name}") as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("w", [5, 7, 8, 13, 20])
def test_balanced_digits_reconstruct(w):
    rng = SplitMix64(20 + w)
    S = 9
    half = 1 << (w - 1)
    vals = [0, 1, -1, half, -half, (1 << (w * S - 1)), -(1 << (w * S - 1))]
    vals += [int(x) - (1 << 62) for x in rng.next(200)]
    vals += [(int(x) << 7) - (1 << (w * S - 2)) for x in rng.next(50) >> np.uint64(64 - w * S + 9)] if w * S - 9 < 64 else []
    for T in vals:
        if abs(T) > (1 << (w * S - 1)):
            continue
        d = slicing.balanced_digits(T, w, S)
        assert sum(x << (w * (S - 1 - p)) for p, x in enumerate(d)) == T
        assert all(-half <= x < half for x in d[1:])
        assert -half <= d[0] <= half


def test_bitfield_digits_reconstruct():
    rng = SplitMix64(3)
    for x in rng.next(100):
        T = int(x) - (1 << 63)
        d = slicing.bitfield_digits(T, 13, 5)
        assert sum(v << (13 * (4 - p)) for p, v in enumerate(d)) == T


def test_fixed_point_truncation_error():
    """0 <= (x - T 2^-F) * sign(x) and |x 2^F - T| < m (each word truncated once)."""
    rng = SplitMix64(31)
    for m in (2, 4, 8):
        X = loguniform_mdouble(rng, m, 1, 40, -10, 10)
        for k in range(40):
            words = X[:, 0, k]
            F = 90
            T = slicing.fixed_point(words, F)
            xs = exact.to_fraction(words) * Fraction(2) ** F
            assert abs(xs - T) < m
            # enough fraction bits: no truncation at all
            Fbig = 53 * m + 1200
            assert slicing.fixed_point(words, Fbig) == exact.to_fraction(words) * Fraction(2) ** Fbig


def test_split_reconstructs_entries_exactly_with_full_coverage():
    """P1: with S w bits covering every word's last bit, the digits times their
    weights sum back to the entry exactly."""
    A, _ = dd_n64()
    sp = slicing.Split(A, w=8, S=16, rows=range(8))
    assert sp.in_range
    for a in range(8):
        for k in range(64):
            v = sum(Fraction(int(sp.digits[p, a, k])) * Fraction(2) ** sp.digit_weight_exponent(a, p)
                    for p in range(16))
            assert v == exact.to_fraction(A[:, a, k])


def test_split_digit_bounds_and_exponents():
    rng = SplitMix64(32)
    X = loguniform_mdouble(rng, 4, 6, 30, -20, 20)
    sp = slicing.Split(X, w=8, S=12)
    assert np.abs(sp.digits).max() <= 128
    for a in range(6):
        E = max(math.frexp(float(X[j, a, k]))[1] for j in range(4) for k in range(30) if X[j, a, k] != 0)
        assert sp.E[a] == E          # frexp exponent == ilogb + 1
        # the leading digit keeps the two headroom bits: |d_0| <= 2^(w-2) + 1
        assert np.abs(sp.digits[0, a]).max() <= 65


def test_split_flags_out_of_range_input():
    """Words that all share the top exponent can sum past 2^(E+1): flagged."""
    X = np.zeros((4, 1, 2))
    X[:, 0, 0] = [1.75, 1.75, 1.75, 1.75]     # not an m-double in normal form
    X[:, 0, 1] = [0.5, 0.0, 0.0, 0.0]
    assert not slicing.Split(X, w=8, S=8).in_range
    X[:, 0, 0] = [1.75, 2.0 ** -60, 0.0, 0.0]
    assert slicing.Split(X, w=8, S=8).in_range


def test_diagonal_sums_brute_force():
    rng = SplitMix64(33)
    A = uniform_mdouble(rng, 2, 3, 5)
    B = uniform_mdouble(rng, 2, 5, 4)
    w, S_A, S_B, D = 7, 6, 5, 8
    sp = slicing.SlicedProduct(A, B, w, S_A, S_B, D)
    for i in range(3):
        for j in range(4):
            for t in range(D):
                s = 0
                for p in range(S_A):
                    q = t - p
                    if 0 <= q < S_B:
                        for k in range(5):
                            s += int(sp.A.digits[p, i, k]) * int(sp.B.digits[q, j, k])
                assert sp.s[t, i, j] == s


def test_diagonal_sums_beyond_int64_brute_force():
    """24-bit digits over a long K: diagonal sums past 2^63 are still exact
    (checked by loops over p, q, k in Python integers)."""
    rng = SplitMix64(34)
    A = uniform_mdouble(rng, 8, 1, 6144)
    B = uniform_mdouble(rng, 8, 6144, 1)
    w, S, D = 24, 19, 20
    sp = slicing.SlicedProduct(A, B, w, S, S, D)
    assert sp.s.dtype == object                      # the int64 bound did not hold
    dA = [[int(x) for x in sp.A.digits[p, 0]] for p in range(S)]
    dB = [[int(x) for x in sp.B.digits[q, 0]] for q in range(S)]
    big = 0
    for t in range(D):
        s = 0
        for p in range(S):
            q = t - p
            if 0 <= q < S:
                s += sum(a * b for a, b in zip(dA[p], dB[q]))
        assert sp.s[t, 0, 0] == s
        big = max(big, abs(s))
    # and the whole method still reaches the rounded exact product
    ex = exact.ExactProduct(A, B, [0], [0])
    assert ex.error_ratio(sp.result()).max() <= 1.0


@pytest.mark.parametrize("m,w", [(2, 8), (2, 7), (4, 8), (2, 20)])
def test_all_pairs_full_coverage_equals_rounded_exact_product(m, w):
    """P3: keeping every pair with S covering every bit, the fused result is the
    greedy rounding of the exact product (computed from mantissas by O2)."""
    rng = SplitMix64(40 + m + w)
    A = uniform_mdouble(rng, m, 5, 9)
    B = uniform_mdouble(rng, m, 9, 6)
    bits = 53 * m + 60
    S = -(-bits // w)
    sp = slicing.SlicedProduct(A, B, w, S, S, 2 * S - 1)
    ex = exact.exact_product_full(A, B)
    for i in range(5):
        for j in range(6):
            assert sp.value(i, j) == ex.exact(i, j)
            assert sp.words(i, j) == exact.greedy_words(ex.exact(i, j), m)


def test_transposed_operands_agree():
    rng = SplitMix64(41)
    A = uniform_mdouble(rng, 2, 4, 6)
    B = uniform_mdouble(rng, 2, 6, 3)
    ref = slicing.SlicedProduct(A, B, 8, 10, 10, 12).result()
    At = np.ascontiguousarray(A.transpose(0, 2, 1))
    Bt = np.ascontiguousarray(B.transpose(0, 2, 1))
    got = slicing.SlicedProduct(At, Bt, 8, 10, 10, 12, transA=True, transB=True).result()
    assert np.array_equal(ref, got)


def test_power_of_two_scaling_commutes():
    rng = SplitMix64(42)
    A = uniform_mdouble(rng, 4, 4, 8)
    B = uniform_mdouble(rng, 4, 8, 4)
    base = slicing.SlicedProduct(A, B, 8, 20, 20, 26).result()
    for k in (-37, 5, 200):
        scaled = slicing.SlicedProduct(A * 2.0 ** k, B, 8, 20, 20, 26).result()
        assert np.array_equal(scaled, base * 2.0 ** k)


def test_truncated_split_error_within_bound():
    """Fewer pieces and a diagonal cut: the result still meets
    |C - C_exact| <= 2K 2^(-52m) |A||B| with the counts the error analysis
    gives (w S >= 52m + range + log2 m + 4 - log2 K; w D >= 52m + 2 ranges + 11
    + log2 S - log2 K)."""
    rng = SplitMix64(43)
    m, n = 2, 24
    A = loguniform_mdouble(rng, m, n, n, -6, 6)
    B = loguniform_mdouble(rng, m, n, n, -6, 6)
    w = 8
    rA = int(slicing.row_exponents(A)[1].max())
    rB = int(slicing.row_exponents(slicing.logical(B, True))[1].max())
    lgK = math.log2(n)
    S_A = math.ceil((52 * m + rA + 1 + 4 - lgK) / w)
    S_B = math.ceil((52 * m + rB + 1 + 4 - lgK) / w)
    S = max(S_A, S_B)
    D = math.ceil((52 * m + rA + rB + 11 + math.log2(S) - lgK) / w)
    sp = slicing.SlicedProduct(A, B, w, S_A, S_B, D)
    assert sp.A.in_range and sp.B.in_range
    ex = exact.exact_product_full(A, B)
    ratio = ex.error_ratio(sp.result())
    assert ratio.max() <= 1.0
    # four digits fewer on each side and eight diagonals fewer: the bound breaks
    worse = slicing.SlicedProduct(A, B, w, S_A - 4, S_B - 4, D - 8)
    assert ex.error_ratio(worse.result()).max() > 1.0


def test_paper_pattern_quarters_have_fixed_exponents():
    """Section 2: the four 13-bit quarters of the 52-bit fraction each begin
    with a 1, so each quarter has the same exponent for every sample."""
    expected = [int(x) for x in read_golden("pattern_quarter_exponents.txt")[0]]
    x = paper_pattern_double(SplitMix64(50), 1000)
    frac = x.view(np.uint64) & np.uint64((1 << 52) - 1)
    for q in range(4):
        field = (frac >> np.uint64(13 * (3 - q))) & np.uint64(0x1FFF)
        val = field.astype(np.float64) * 2.0 ** (-13 * (q + 1))   # quarter q of the fraction
        ex = np.frexp(val)[1]
        assert (ex == expected[q]).all()
        assert ((field >> np.uint64(12)) == 1).all()


def test_paper_pattern_diagonal_sums_are_exact_in_double():
    """Section 2: with the pattern data the quarter products of a double-double
    inner product of length 6,144 sum exactly in double arithmetic."""
    rng = SplitMix64(51)
    n = 6144
    X = paper_pattern_mdouble(rng, 2, 1, n)
    Y = paper_pattern_mdouble(rng, 2, 1, n)

    def quarters(words):
        out = []
        for j in range(2):
            bits = words[j].view(np.uint64)
            frac = (bits & np.uint64((1 << 52) - 1)) | np.uint64(1 << 52)
            e = ((bits >> np.uint64(52)).astype(np.int64) - 1023 - 52)
            for q in range(4):
                sh = 13 * (3 - q)
                field = (frac >> np.uint64(sh)) & np.uint64(0x3FFF if q == 0 else 0x1FFF)
                out.append(field.astype(np.float64) * np.exp2((e + sh).astype(np.float64)))
        return out

    xq = quarters(X[:, 0, :])
    yq = quarters(Y[:, 0, :])
    for k in range(0, n, 997):
        assert sum(Fraction(float(q[k])) for q in xq) == exact.to_fraction(X[:, 0, k])
    for i in range(8):
        s_double = 0.0
        s_exact = Fraction(0)
        for j in range(i + 1):
            s_double += float(np.dot(xq[j], yq[i - j]))
            s_exact += sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(xq[j], yq[i - j]))
        assert Fraction(s_double) == s_exact


def test_group_values_recombine_to_the_fused_integer():
    """The 64-bit group sums the wide GPU mode stores recombine, with weights
    2^(w (D-1-t1)), to the fused integer X, which the full-coverage test pins to
    the exact product; one group spanning every diagonal is X itself."""
    rng = SplitMix64(44)
    A, B = uniform_mdouble(rng, 2, 3, 40), uniform_mdouble(rng, 2, 40, 2)
    w, S, D = 8, 16, 24
    sp = slicing.SlicedProduct(A, B, w, S, S, D)
    for group in (1, 3, 5, D):
        bounds = [(g * group, min(D, (g + 1) * group) - 1) for g in range(-(-D // group))]
        for a in range(3):
            for b in range(2):
                V = slicing.group_values(sp.s[:, a, b], w, bounds)
                X = sum(v << (w * (D - 1 - t1)) for v, (_, t1) in zip(V, bounds))
                assert X == slicing.fuse_integer(sp.s[:, a, b], w, D)
                if group == D:
                    assert V == [X]
