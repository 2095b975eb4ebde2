"""The adjoint: mw_gemm_backward and the MWGemm autograd function.

For C = A B and L = sum(C * W), dL/dA = W B^T and dL/dB = A^T W exactly (L is
bilinear).  The library's gradients are checked against the oracle's exact
products on sampled entries (bound 2K 2^(-52m) |.||.| of each product) and, on
the double-double case of 2048 x 1024 x 2048, against central finite
differences of L evaluated in quad-double with the library's own m = 4 product.
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

from conftest import record_worst, to_dev
from oracle import exact
from synthetic import SplitMix64, adjoint_case, uniform_mdouble

pytestmark = pytest.mark.gpu


def as_mdouble(W, m):
    out = np.zeros((m,) + W.shape)
    out[0] = W
    return out


def check_entries(grad, X, Y, entries, m):
    """grad[:, i, j] against the exact (X Y)_ij and its bound."""
    rows = sorted({i for i, _ in entries})
    cols = sorted({j for _, j in entries})
    ex = exact.ExactProduct(X, Y, rows, cols)
    worst = 0.0
    for i, j in entries:
        a, b = rows.index(i), cols.index(j)
        err = abs(exact.to_fraction(grad[:, i, j]) - ex.exact(a, b))
        bnd = ex.bound(a, b)
        assert err <= bnd, (i, j)
        worst = max(worst, float(err / bnd) if bnd else 0.0)
    return worst


@pytest.mark.parametrize("mode", ["ozaki", "plain"])
def test_backward_small_against_exact(mw, cuda, mode):
    rng = SplitMix64(500)
    M, K, N = 37, 50, 29
    A, B = uniform_mdouble(rng, 2, M, K), uniform_mdouble(rng, 2, K, N)
    G = uniform_mdouble(rng, 2, M, N)
    dA, dB = mw.mw_gemm_backward(to_dev(A, cuda), to_dev(B, cuda), to_dev(G, cuda), mode=mode)
    dA, dB = dA.cpu().numpy(), dB.cpu().numpy()
    BT = np.ascontiguousarray(B.transpose(0, 2, 1))
    AT = np.ascontiguousarray(A.transpose(0, 2, 1))
    assert exact.exact_product_full(G, BT).error_ratio(dA).max() <= 1.0
    assert exact.exact_product_full(AT, G).error_ratio(dB).max() <= 1.0


def test_autograd_function(mw, cuda):
    rng = SplitMix64(501)
    A = to_dev(uniform_mdouble(rng, 2, 20, 30), cuda).requires_grad_(True)
    B = to_dev(uniform_mdouble(rng, 2, 30, 25), cuda).requires_grad_(True)
    W = rng.sym(20 * 25).reshape(20, 25)
    Wmd = to_dev(as_mdouble(W, 2), cuda)
    C = mw.MWGemm.apply(A, B)
    loss = (C * Wmd).sum()            # dloss/dC = the m-double W (planes W, 0)
    loss.backward()
    An, Bn = A.detach().cpu().numpy(), B.detach().cpu().numpy()
    Wn = as_mdouble(W, 2)
    gA = exact.exact_product_full(Wn, np.ascontiguousarray(Bn.transpose(0, 2, 1)))
    gB = exact.exact_product_full(np.ascontiguousarray(An.transpose(0, 2, 1)), Wn)
    assert gA.error_ratio(A.grad.cpu().numpy()).max() <= 1.0
    assert gB.error_ratio(B.grad.cpu().numpy()).max() <= 1.0


def qd_loss_row(mw, cuda, a_row, tB4, w_row):
    """sum_n w_n (a_row B)_n in quad double with the library's m = 4 product
    (tB4: B padded to four words, on the device)."""
    K, N = tB4.shape[1], tB4.shape[2]
    a4 = np.zeros((4, 1, K)); a4[:a_row.shape[0], 0, :] = a_row
    c = mw.mw_gemm(to_dev(a4, cuda), tB4, mode="ozaki")                      # 1 x N
    w4 = np.zeros((4, N, 1)); w4[0, :, 0] = w_row
    L = mw.mw_gemm(c, to_dev(w4, cuda), mode="ozaki").cpu().numpy()          # 1 x 1
    return exact.to_fraction(L[:, 0, 0])


@pytest.mark.slow
def test_adjoint_case_2048(mw, cuda):
    """A 2048 x 1024, B 1024 x 2048 double doubles, W 2048 x 2048, seed 4:
    forward through the Ozaki form, dA and dB from the autograd function,
    64 sampled entries against the exact gradient and against quad-double
    central differences with h = 2^-20.  The exact gradient (the oracle's
    rational products W B^T and A^T W) is the independent check; the central
    differences evaluate the loss with this library's own quad-double product,
    so they confirm the gradient's meaning but are not independent of it."""
    A, B, W = adjoint_case()
    tA = to_dev(A, cuda).requires_grad_(True)
    tB = to_dev(B, cuda).requires_grad_(True)
    Wmd = as_mdouble(W, 2)
    C = mw.MWGemm.apply(tA, tB)
    (C * to_dev(Wmd, cuda)).sum().backward()
    dA, dB = tA.grad.cpu().numpy(), tB.grad.cpu().numpy()
    rng = SplitMix64(504)
    M, K = A.shape[1], A.shape[2]
    N = B.shape[2]
    ea = [(int(i), int(j)) for i, j in zip(rng.next(32) % np.uint64(M), rng.next(32) % np.uint64(K))]
    eb = [(int(i), int(j)) for i, j in zip(rng.next(32) % np.uint64(K), rng.next(32) % np.uint64(N))]
    BT = np.ascontiguousarray(B.transpose(0, 2, 1))
    AT = np.ascontiguousarray(A.transpose(0, 2, 1))
    record_worst("dd adjoint dA = W B^T, 32 sampled entries", check_entries(dA, Wmd, BT, ea, 2))
    record_worst("dd adjoint dB = A^T W, 32 sampled entries", check_entries(dB, AT, Wmd, eb, 2))
    # central differences in quad double: L is bilinear, so (L(+h) - L(-h)) / 2h is the
    # derivative up to the quad-double rounding of the two loss values
    h = Fraction(2) ** -20
    exA = exact.ExactProduct(Wmd, BT, sorted({i for i, _ in ea}), sorted({j for _, j in ea}))
    exB = exact.ExactProduct(AT, Wmd, sorted({k for k, _ in eb}), sorted({n for _, n in eb}))
    A4 = np.zeros((4, M, K)); A4[:2] = A
    tA4 = to_dev(A4, cuda)
    B4 = np.zeros((4, K, N)); B4[:2] = B
    tB4 = to_dev(B4, cuda)
    for i, j in ea:
        vals = []
        for sgn in (1, -1):
            v = exact.to_fraction(A[:, i, j]) + sgn * h
            a_row = np.vstack([A[:, i, :], np.zeros((2, K))])
            a_row[:, j] = exact.greedy_words(v, 4)
            vals.append(qd_loss_row(mw, cuda, a_row, tB4, W[i]))
        fd = (vals[0] - vals[1]) / (2 * h)
        a, b = exA.rows.index(i), exA.cols.index(j)
        assert abs(fd - exA.exact(a, b)) <= exA.bound(a, b) * Fraction(2) ** -90
        assert abs(exact.to_fraction(dA[:, i, j]) - fd) <= exA.bound(a, b) * (1 + Fraction(2) ** -80)
    for k, n in eb:
        vals = []
        for sgn in (1, -1):
            v = exact.to_fraction(B[:, k, n]) + sgn * h
            b_col = np.vstack([B[:, :, n], np.zeros((2, K))])
            b_col[:, k] = exact.greedy_words(v, 4)
            Ab = mw.mw_gemm(tA4, to_dev(np.ascontiguousarray(b_col[:, :, None]), cuda), mode="ozaki")
            w4 = np.zeros((4, 1, M)); w4[0, 0, :] = W[:, n]
            L = mw.mw_gemm(to_dev(w4, cuda), Ab, mode="ozaki").cpu().numpy()
            vals.append(exact.to_fraction(L[:, 0, 0]))
        fd = (vals[0] - vals[1]) / (2 * h)
        a, b = exB.rows.index(k), exB.cols.index(n)
        assert abs(fd - exB.exact(a, b)) <= exB.bound(a, b) * Fraction(2) ** -90
        assert abs(exact.to_fraction(dB[:, k, n]) - fd) <= exB.bound(a, b) * (1 + Fraction(2) ** -80)
