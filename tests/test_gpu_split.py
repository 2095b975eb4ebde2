"""mw_split on the GPU against the oracle's pieces, bit for bit."""
import numpy as np
import pytest
import torch

from conftest import to_dev
from oracle import slicing
from synthetic import SplitMix64, loguniform_mdouble, paper_pattern_mdouble, uniform_mdouble

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [2, 4, 8])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("fmt,w", [("bf16", 8), ("bf16", 7), ("f64", 20)])
def test_pieces_bit_exact(mw, cuda, m, trans, fmt, w):
    rng = SplitMix64(200 + m + 3 * w + int(trans))
    R, K = 37, 101                                    # ragged: neither a multiple of 32 nor 64
    L = loguniform_mdouble(rng, m, R, K, -12, 12)
    L[:, 3, :] = 0.0                                  # an all-zero row
    L[:, 5, 7] = 0.0                                  # a zero entry
    X = np.ascontiguousarray(L.transpose(0, 2, 1)) if trans else L
    S = -(-(52 * m + 30) // w)
    digits, exps, spread = mw.mw_split(to_dev(X, cuda), w, S, trans=trans, fmt=fmt)
    mw.check_status()
    ref = slicing.Split(L, w, S)
    got = digits.to(torch.float64).cpu().numpy()
    assert got.shape[2] % 64 == 0 and not got[:, :, K:].any()
    assert np.array_equal(got[:, :, :K].astype(np.int64), ref.digits)
    assert np.array_equal(exps.cpu().numpy(), ref.E)
    assert np.array_equal(spread.cpu().numpy(), ref.range)


def test_paper_pattern_pieces(mw, cuda):
    rng = SplitMix64(210)
    L = paper_pattern_mdouble(rng, 2, 16, 64)
    digits, exps, _ = mw.mw_split(to_dev(L, cuda), 8, 16)
    ref = slicing.Split(L, 8, 16)
    assert np.array_equal(digits.to(torch.float64).cpu().numpy()[:, :, :64].astype(np.int64),
                          ref.digits)


def test_status_nonfinite_and_range(mw, cuda):
    mw.get_status(clear=True)
    X = uniform_mdouble(SplitMix64(211), 2, 4, 8)
    X[0, 1, 2] = np.inf
    mw.mw_split(to_dev(X, cuda), 8, 16)
    assert mw.get_status(clear=True) & mw.MW_ENONFINITE
    Y = np.zeros((4, 1, 8))
    Y[:, 0, 0] = 1.75                                 # four equal words: not normalised
    mw.mw_split(to_dev(Y, cuda), 8, 8)
    assert mw.get_status(clear=True) & mw.MW_ERANGE
    mw.mw_split(to_dev(uniform_mdouble(SplitMix64(212), 4, 3, 8), cuda), 8, 30)
    assert mw.get_status(clear=True) == 0
