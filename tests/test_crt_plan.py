"""The residue form's host side on the CPU: the library's table of moduli
(pairwise coprime, balanced residues within bfloat16's exact integers, the
drain chunk of every modulus keeping fp32 sums exact) and the planner (enough
fixed-point bits for the bound, enough moduli for an exact reconstruction),
checked with the oracle's own arithmetic; and the oracle run with the planner's
counts meets the bound."""
import math

import numpy as np
import pytest

from oracle import crt, exact, slicing
from synthetic import SplitMix64, loguniform_mdouble


def test_moduli_table(mw):
    ps = mw.crt_moduli()
    assert len(ps) >= 90 and len(set(ps)) == len(ps)
    assert crt.pairwise_coprime(ps)
    assert all(2 < p <= 513 and p % 2 == 1 for p in ps)   # odd: no halfway sums
    # every balanced residue is an integer bfloat16 holds exactly
    assert max(p // 2 for p in ps) <= 256
    # the bits a plan can reach with the whole table
    assert math.log2(crt.modulus_product(ps)) > 700
    assert mw.crt_moduli(5) == ps[:5]


@pytest.mark.parametrize("m", [2, 4])
def test_crt_plan_constraints(mw, m):
    ps = mw.crt_moduli()
    for K in (1, 7, 64, 1024, 4096, 40000):
        for ra, rb in ((0, 0), (16, 16), (40, 40), (3, 60)):
            p = mw.mw_plan_gemm(m, "crt", 100, 100, K, ra, rb)
            assert p.mode == mw.MW_CRT and p.w == 1 and p.group == 1
            lgK = math.log2(K)
            assert p.S_A >= 52 * m + ra + math.log2(m) + 5 - lgK - 1e-9
            assert p.S_B >= 52 * m + rb + math.log2(m) + 5 - lgK - 1e-9
            # the fewest moduli whose product exceeds 8 K 2^(L_A + L_B - 2)
            need = 8 * K * 2 ** (p.S_A + p.S_B - 2)
            assert crt.modulus_product(ps[:p.D]) > need
            assert crt.modulus_product(ps[:p.D - 1]) <= need


def test_crt_plan_rejects(mw):
    for m in (8, 16):
        with pytest.raises(mw.MWError):
            mw.mw_plan_gemm(m, "crt", 10, 10, 10, 0, 0)
    with pytest.raises(mw.MWError):                     # more bits than the table holds
        mw.mw_plan_gemm(4, "crt", 10, 10, 10, 300, 300)


@pytest.mark.parametrize("m,lo,hi", [(2, -20, 20), (4, -8, 8)])
def test_oracle_with_planner_counts_meets_bound(mw, m, lo, hi):
    rng = SplitMix64(960 + m)
    M, N, K = 5, 4, 64
    A, B = loguniform_mdouble(rng, m, M, K, lo, hi), loguniform_mdouble(rng, m, K, N, lo, hi)
    rA = int(slicing.row_exponents(A)[1].max())
    rB = int(slicing.row_exponents(np.ascontiguousarray(B.transpose(0, 2, 1)))[1].max())
    p = mw.mw_plan_gemm(m, "crt", M, N, K, rA, rB)
    rp = crt.ResidueProduct(A, B, p.S_A, p.S_B, mw.crt_moduli(p.D))
    for a in range(M):
        for b in range(N):
            assert rp.X(a, b) == rp.X_direct(a, b)
    assert exact.exact_product_full(A, B).error_ratio(rp.result()).max() <= 1.0
