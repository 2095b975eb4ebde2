"""Pins of the residue oracle (oracle/crt.py) against what mathematics fixes:
the Chinese remainder theorem by brute force, the exact integer products
computed directly, the slice form with every pair kept (itself pinned to the
exact product), the exact product's error bound, and closed forms."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import crt, exact, slicing
from synthetic import SplitMix64, loguniform_mdouble, paper_pattern_mdouble, uniform_mdouble


def primes_from(lo, count):
    """The first `count` primes >= lo (trial division; small numbers only)."""
    out, n = [], max(lo, 2)
    while len(out) < count:
        if all(n % d for d in range(2, math.isqrt(n) + 1)):
            out.append(n)
        n += 1
    return out


def moduli_for_bits(bits, lo=200):
    ps = []
    for p in primes_from(lo, 400):
        ps.append(p)
        if math.log2(crt.modulus_product(ps)) > bits:
            return ps
    raise AssertionError("not enough primes")


def test_balanced_residue_range_and_congruence():
    rng = np.random.default_rng(0)
    for p in (2, 3, 256, 257, 362, 363, 512, 513):
        lo, hi = -(p // 2), (p + 1) // 2 - 1
        for x in list(rng.integers(-10 ** 18, 10 ** 18, 200)) + [0, 1, -1, p, -p, p // 2, -(p // 2)]:
            r = crt.balanced_residue(int(x), p)
            assert lo <= r <= hi and (int(x) - r) % p == 0, (x, p, r)
        assert max(abs(crt.balanced_residue(x, p)) for x in range(p)) == p // 2
    # a residue of p <= 513 is an integer bfloat16 holds exactly (|r| <= 256)
    assert all(abs(crt.balanced_residue(x, 513)) <= 256 for x in range(-600, 600))


def test_crt_reconstruct_brute_force_small():
    """Moduli 4, 9, 5, 7: every integer in (-P/2, P/2] comes back from its residues."""
    moduli = [4, 9, 5, 7]
    assert crt.pairwise_coprime(moduli)
    P = crt.modulus_product(moduli)
    for x in range(-P // 2 + 1, P // 2 + 1):
        ys = [crt.balanced_residue(x, p) for p in moduli]
        assert crt.crt_reconstruct(ys, moduli) == x
    # outside the range the reconstruction wraps by P: the bound on |X| matters
    x = P // 2 + 3
    assert crt.crt_reconstruct([x % p for p in moduli], moduli) == x - P


def test_crt_reconstruct_large_random():
    moduli = primes_from(257, 70)
    P = crt.modulus_product(moduli)
    rng = SplitMix64(900)
    for u in rng.next(50):
        x = ((int(u) * P) >> 64) - P // 2 + 1              # spread over (-P/2, P/2]
        ys = [crt.balanced_residue(x, p) for p in moduli]
        assert crt.crt_reconstruct(ys, moduli) == x
    assert not crt.pairwise_coprime([6, 35, 9])


@pytest.mark.parametrize("m,M,N,K,lo,hi,seed", [
    (2, 5, 4, 7, None, None, 1),
    (2, 6, 3, 33, -10, 10, 2),
    (4, 3, 5, 20, -8, 8, 3),
    (4, 4, 4, 1, -3, 3, 4),
])
def test_residue_product_equals_direct_integer_product(m, M, N, K, lo, hi, seed):
    rng = SplitMix64(910 + seed)
    if lo is None:
        A, B = uniform_mdouble(rng, m, M, K), uniform_mdouble(rng, m, K, N)
    else:
        A, B = loguniform_mdouble(rng, m, M, K, lo, hi), loguniform_mdouble(rng, m, K, N, lo, hi)
    L_A = crt.fixed_point_bits(m, K, 20)
    L_B = crt.fixed_point_bits(m, K, 20)
    moduli = moduli_for_bits(crt.product_bits_needed(L_A, L_B, K))
    rp = crt.ResidueProduct(A, B, L_A, L_B, moduli)
    assert rp.A.in_range and rp.B.in_range
    for a in range(M):
        for b in range(N):
            assert rp.X(a, b) == rp.X_direct(a, b)
            for i, p in enumerate(moduli):                 # each Y_i is congruent to X
                assert (int(rp.Y[i, a, b]) - rp.X(a, b)) % p == 0


def test_too_few_moduli_break_the_reconstruction():
    """With P below 2 max|X| some reconstructed product differs from the direct one."""
    rng = SplitMix64(920)
    A, B = uniform_mdouble(rng, 2, 4, 30), uniform_mdouble(rng, 2, 30, 4)
    L = crt.fixed_point_bits(2, 30, 4)
    need = crt.product_bits_needed(L, L, 30)
    short = moduli_for_bits(need - 40)
    rp = crt.ResidueProduct(A, B, L, L, short)
    assert any(rp.X(a, b) != rp.X_direct(a, b) for a in range(4) for b in range(4))


@pytest.mark.parametrize("m,w,S_A,S_B", [(2, 8, 15, 16), (4, 8, 26, 25), (2, 7, 18, 18)])
def test_residue_form_equals_slice_form_with_every_pair(m, w, S_A, S_B):
    """With L = w S the residue form computes the same integer as the slice form
    keeping every pair (D = S_A + S_B - 1), which the slice pins tie to the exact
    product: the words agree bit for bit."""
    rng = SplitMix64(930 + m + w)
    A, B = loguniform_mdouble(rng, m, 5, 40, -6, 6), loguniform_mdouble(rng, m, 40, 6, -6, 6)
    L_A, L_B = w * S_A, w * S_B
    moduli = moduli_for_bits(crt.product_bits_needed(L_A, L_B, 40))
    rp = crt.ResidueProduct(A, B, L_A, L_B, moduli)
    sp = slicing.SlicedProduct(A, B, w, S_A, S_B, S_A + S_B - 1)
    assert np.array_equal(rp.result(), sp.result())
    for a in range(5):
        for b in range(6):
            assert rp.value(a, b) == sp.value(a, b)


@pytest.mark.parametrize("m,kind", [(2, "uniform"), (2, "log20"), (4, "log20"), (4, "pattern"),
                                    (2, "adversarial")])
def test_residue_form_within_the_bound(m, kind):
    rng = SplitMix64(940 + m)
    M, N, K = 4, 5, 48
    if kind == "uniform":
        A, B = uniform_mdouble(rng, m, M, K), uniform_mdouble(rng, m, K, N)
    elif kind == "log20":
        A, B = loguniform_mdouble(rng, m, M, K, -20, 20), loguniform_mdouble(rng, m, K, N, -20, 20)
    elif kind == "pattern":
        A, B = paper_pattern_mdouble(rng, m, M, K), paper_pattern_mdouble(rng, m, K, N)
    else:   # tiny entries of A meeting large entries of B and the other way round
        A, B = uniform_mdouble(rng, m, M, K), uniform_mdouble(rng, m, K, N)
        A[:, :, ::2] *= 2.0 ** -30
        B[:, 1::2, :] *= 2.0 ** -30
    LA = np.ascontiguousarray(A)
    LB = np.ascontiguousarray(B.transpose(0, 2, 1))
    rA = int(slicing.row_exponents(LA)[1].max())
    rB = int(slicing.row_exponents(LB)[1].max())
    L_A, L_B = crt.fixed_point_bits(m, K, rA), crt.fixed_point_bits(m, K, rB)
    moduli = moduli_for_bits(crt.product_bits_needed(L_A, L_B, K))
    C = crt.ResidueProduct(A, B, L_A, L_B, moduli).result()
    ratio = exact.exact_product_full(A, B).error_ratio(C)
    assert ratio.max() <= 1.0
    # fewer fixed-point bits than the analysis asks for break the bound somewhere
    # (log-uniform rows leave most entries far above their row's smallest one)
    d = 56 if kind == "log20" else 24
    Cs = crt.ResidueProduct(A, B, L_A - d, L_B - d, moduli).result()
    assert exact.exact_product_full(A, B).error_ratio(Cs).max() > 1.0


def test_closed_forms():
    """B = I gives C = A exactly once L covers every bit of A; scaling A by 2^s
    scales C by 2^s bit for bit; K = 1 is the exact product of two m-doubles
    rounded greedily."""
    rng = SplitMix64(950)
    m, n = 2, 6
    A = uniform_mdouble(rng, m, n, n)
    I = np.zeros((m, n, n)); I[0] = np.eye(n)
    L = 200                                   # covers the ~160 bits of a double double
    moduli = moduli_for_bits(crt.product_bits_needed(L, L, n))
    rp = crt.ResidueProduct(A, I, L, L, moduli)
    for a in range(n):
        for b in range(n):
            assert rp.value(a, b) == exact.to_fraction(A[:, a, b])
    B = uniform_mdouble(rng, m, n, n)
    L2 = crt.fixed_point_bits(m, n, 3)
    mod2 = moduli_for_bits(crt.product_bits_needed(L2, L2, n))
    C1 = crt.ResidueProduct(A, B, L2, L2, mod2).result()
    C2 = crt.ResidueProduct(A * 2.0 ** 37, B * 2.0 ** -5, L2, L2, mod2).result()
    assert np.array_equal(C1 * 2.0 ** 32, C2)
    a = uniform_mdouble(rng, 4, 1, 1)
    b = uniform_mdouble(rng, 4, 1, 1)
    L3 = 260
    c = crt.ResidueProduct(a, b, L3, L3, moduli_for_bits(crt.product_bits_needed(L3, L3, 1)))
    want = exact.to_fraction(a[:, 0, 0]) * exact.to_fraction(b[:, 0, 0])
    assert c.value(0, 0) == want
    assert c.words(0, 0) == exact.greedy_words(want, 4)
