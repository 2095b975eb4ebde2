"""mw_elementwise (Table 1's m-double add, mul and div entry by entry) on the GPU
against the textbook oracle's same operations in C: bit for bit, over a ragged
number of entries and magnitudes spread across 2^[-20, 20); division also
within 2^(1-52m) |a / b| of the exact quotient on sampled entries."""
from fractions import Fraction

import numpy as np
import pytest
import torch

from conftest import to_dev
from oracle import textbook
from synthetic import SplitMix64, loguniform_mdouble

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    return textbook.TextbookC()


@pytest.mark.parametrize("m", [2, 4, 8])
@pytest.mark.parametrize("op", ["add", "mul", "div"])
def test_elementwise_bit_exact(mw, cuda, tc, m, op):
    rng = SplitMix64(1100 + 10 * m + len(op))
    n = 70001                                   # not a multiple of the 256-entry blocks
    A = loguniform_mdouble(rng, m, 1, n, -20, 20).reshape(m, n)
    B = loguniform_mdouble(rng, m, 1, n, -20, 20).reshape(m, n)
    C = mw.mw_elementwise(op, to_dev(A, cuda), to_dev(B, cuda)).cpu().numpy()
    assert np.array_equal(C, tc.elementwise(op, A, B))
    if op == "div":
        for e in range(0, n, n // 40):
            q = sum(Fraction(float(x)) for x in A[:, e]) / sum(Fraction(float(x)) for x in B[:, e])
            got = sum(Fraction(float(x)) for x in C[:, e])
            assert abs(got - q) <= Fraction(2) ** (1 - 52 * m) * abs(q), e


def test_elementwise_shapes_and_errors(mw, cuda, tc):
    """Any (m, ...) shape is one run of entries; one entry; a preallocated C; a
    non-contiguous operand or an unknown operation is refused; C may be A."""
    rng = SplitMix64(1150)
    A = loguniform_mdouble(rng, 4, 3, 5, -4, 4)
    B = loguniform_mdouble(rng, 4, 3, 5, -4, 4)
    C = torch.empty((4, 3, 5), dtype=torch.float64, device=cuda)
    out = mw.mw_elementwise("div", to_dev(A, cuda), to_dev(B, cuda), C)
    assert out is C
    assert np.array_equal(C.cpu().numpy(), tc.elementwise("div", A, B))
    one = mw.mw_elementwise("mul", to_dev(A[:, :1, :1], cuda), to_dev(B[:, :1, :1], cuda))
    assert np.array_equal(one.cpu().numpy(), tc.elementwise("mul", A[:, :1, :1], B[:, :1, :1]))
    with pytest.raises(mw.MWError):
        mw.mw_elementwise("add", to_dev(A, cuda).transpose(1, 2), to_dev(B, cuda).transpose(1, 2))
    with pytest.raises(mw.MWError):
        mw.mw_elementwise("pow", to_dev(A, cuda), to_dev(B, cuda))
    tA = to_dev(A, cuda)                        # in place: C is A
    mw.mw_elementwise("add", tA, to_dev(B, cuda), tA)
    assert np.array_equal(tA.cpu().numpy(), tc.elementwise("add", A, B))
