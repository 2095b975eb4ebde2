"""Failure detection without a GPU fault: a bounded wait (the one every
pipeline kernel uses) is made to run out on a barrier that nothing completes;
the kernel raises MW_ETIMEOUT and returns, and the context stays usable."""
import numpy as np
import pytest

from conftest import to_dev
from oracle import slicing
from synthetic import SplitMix64, uniform_mdouble

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports(mw, cuda):
    bits = mw.selftest_timeout(20000)              # 20 ms
    assert bits & mw.MW_ETIMEOUT
    # the context is still usable: a product afterwards is exact and clean
    rng = SplitMix64(800)
    A, B = uniform_mdouble(rng, 2, 33, 40), uniform_mdouble(rng, 2, 40, 27)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, "ozaki")
    C = mw.mw_gemm(tA, tB, plan).cpu().numpy()
    sp = slicing.SlicedProduct(A, B, plan.w, plan.S_A, plan.S_B, plan.D)
    assert np.array_equal(C, sp.result())
    assert mw.get_status(clear=True) == 0


def test_bounded_wait_rejects_bad_limits(mw, cuda):
    with pytest.raises(mw.MWError):
        mw.selftest_timeout(0)
