"""The autotuner on the GPU: it times every admissible candidate on the
caller's operands, caches the fastest per shape class, and the product with
the tuned plan is bit for bit the oracle's for that plan (and within the
bound); a second product of the class re-uses the cache without timing."""
import numpy as np
import pytest

from conftest import to_dev
from oracle import crt, exact, slicing
from synthetic import SplitMix64, loguniform_mdouble

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,M,N,K", [(2, 96, 80, 300), (4, 130, 70, 200), (8, 40, 36, 64)])
def test_tuned_plan_bit_exact(mw, cuda, tmp_path, m, M, N, K):
    from paper_2606_20863_gb300 import autotune
    rng = SplitMix64(1500 + m)
    A, B = loguniform_mdouble(rng, m, M, K, -6, 6), loguniform_mdouble(rng, m, K, N, -6, 6)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    tuner = autotune.Autotuner(str(tmp_path / "t.json"), reps=2)
    plan = tuner.plan_for(tA, tB)
    times = tuner.last
    assert times and len(times) == len(autotune.candidates(m, M, N, K, plan.range_A,
                                                           plan.range_B))
    assert all(t > 0 for t in times.values())
    C = mw.mw_gemm(tA, tB, plan).cpu().numpy()
    if plan.mode == mw.MW_CRT:
        want = crt.ResidueProduct(A, B, plan.S_A, plan.S_B, mw.crt_moduli(plan.D)).result()
    else:
        want = slicing.SlicedProduct(A, B, plan.w, plan.S_A, plan.S_B, plan.D).result()
    assert np.array_equal(C, want)
    assert exact.exact_product_full(A, B).error_ratio(C).max() <= 1.0
    # same class (ragged shape inside the same power-of-two buckets): no timing
    tuner.last = None
    A2, B2 = A[:, :M - 1, :K - 5], B[:, :K - 5, :N - 1]
    assert autotune.shape_key(m, M - 1, N - 1, K - 5, 0, 0) == autotune.shape_key(m, M, N, K, 0, 0)
    tA2, tB2 = to_dev(A2, cuda), to_dev(B2, cuda)
    p2 = tuner.plan_for(tA2, tB2)
    if (p2.range_A, p2.range_B) == (plan.range_A, plan.range_B):
        assert tuner.last is None and (p2.mode, p2.w, p2.chunk) == (plan.mode, plan.w, plan.chunk)
