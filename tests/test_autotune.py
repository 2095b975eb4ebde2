"""The autotuner's host logic on the CPU: every candidate it would time meets
the bound (the planner's shares of 2K 2^(-52m), exact drains, enough moduli),
inadmissible plans are refused, the fastest admissible choice is cached per
shape class and read back, and a cached choice re-plans for the exact shape."""
import json

import pytest

from oracle import crt, slicing
from synthetic import SplitMix64, loguniform_mdouble


@pytest.fixture
def tuner(mw, tmp_path):
    from paper_2606_20863_gb300 import autotune
    return autotune, autotune.Autotuner(str(tmp_path / "tune.json"))


@pytest.mark.parametrize("m,K,r", [(2, 4096, 40), (4, 1024, 16), (8, 128, 0), (16, 64, 3)])
def test_candidates_are_admissible(tuner, m, K, r):
    at, _ = tuner
    cs = at.candidates(m, 512, 512, K, r, r)
    assert cs and all(at.admissible(at.plan_of(c, m, 512, 512, K, r, r), K) for c in cs)
    assert any(c.form == "crt" for c in cs) == (m in (2, 4))
    assert {c.w for c in cs if c.form == "ozaki"} == {6, 7, 8}


def test_inadmissible_plans_are_refused(mw, tuner):
    at, _ = tuner
    p = mw.mw_plan_gemm(4, "ozaki", 64, 64, 1024, 10, 10)
    assert at.admissible(p, 1024)
    p.chunk = 2 * ((1 << 24) >> (2 * p.w - 2))          # fp32 sums no longer exact
    assert not at.admissible(p, 1024)
    p = mw.mw_plan_gemm(4, "ozaki", 64, 64, 1024, 10, 10)
    p.S_A -= 2                                          # truncation beyond its share
    assert not at.admissible(p, 1024)
    q = mw.mw_plan_gemm(2, "crt", 64, 64, 1024, 10, 10)
    assert at.admissible(q, 1024)
    q.D -= 3                                            # too few moduli
    assert not at.admissible(q, 1024)


def test_choice_cached_and_replanned(mw, tuner, tmp_path):
    at, t = tuner
    # a fake timing: the residue form is fastest, then wider pieces
    def fake(p):
        return 1.0 if p.mode == mw.MW_CRT else 10.0 - p.w + p.chunk / 1e6
    choice, times = t.choose(4, 1000, 1000, 1000, 16, 16, fake)
    assert choice == at.Choice("crt") and len(times) >= 5
    key = at.shape_key(4, 1000, 1000, 1000, 16, 16)
    assert key == "m4/M1024/N1024/K1024/rA16/rB16"
    again = at.Autotuner(t.path)
    assert again.cached(key) == choice
    stored = json.load(open(t.path))[key]
    assert stored["form"] == "crt" and "ms" in stored
    # slices only (m = 8): the fastest width wins
    c8, _ = t.choose(8, 100, 100, 100, 0, 0, fake)
    assert c8.form == "ozaki" and c8.w == 8
    p = at.plan_of(c8, 8, 90, 70, 120, 0, 0)            # same class, exact shape
    assert p.m == 8 and p.w == 8 and at.admissible(p, 120)


def test_tuned_slice_plans_meet_the_bound_on_the_oracle(mw, tuner):
    """Every slice candidate's plan, run by the oracle, meets the bound (w = 6, 7, 8)."""
    at, _ = tuner
    from oracle import exact
    rng = SplitMix64(1400)
    A, B = loguniform_mdouble(rng, 2, 4, 48, -8, 8), loguniform_mdouble(rng, 2, 48, 5, -8, 8)
    import numpy as np
    rA = int(slicing.row_exponents(A)[1].max())
    rB = int(slicing.row_exponents(np.ascontiguousarray(B.transpose(0, 2, 1)))[1].max())
    for c in at.candidates(2, 4, 5, 48, rA, rB):
        p = at.plan_of(c, 2, 4, 5, 48, rA, rB)
        if c.form == "crt":
            C = crt.ResidueProduct(A, B, p.S_A, p.S_B, mw.crt_moduli(p.D)).result()
        else:
            C = slicing.SlicedProduct(A, B, p.w, p.S_A, p.S_B, p.D).result()
        assert exact.exact_product_full(A, B).error_ratio(C).max() <= 1.0, c
