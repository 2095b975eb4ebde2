"""mw_gemm on the GPU against the oracle.

MW_OZAKI: the integer partial sums of every diagonal group and the final
words match the oracle's error-free summation bit for bit; the words meet the
componentwise bound against the exact product.  MW_PLAIN: its diagonal sums
are exact, its m-double fusion is checked against the oracle's exact fused
value and against the bound.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

from conftest import record_worst, to_dev
from oracle import exact, slicing
from synthetic import (SplitMix64, dd_n64, loguniform_mdouble, loguniform_pair, uniform_mdouble)

pytestmark = pytest.mark.gpu


def logical_pair(A, B, transA, transB):
    LA = np.ascontiguousarray(A.transpose(0, 2, 1)) if transA else A
    LB = np.ascontiguousarray(B.transpose(0, 2, 1)) if transB else B
    return LA, LB


def run(mw, dev, A, B, plan, transA=False, transB=False):
    tA, tB = to_dev(A, dev), to_dev(B, dev)
    m, M, N, K = mw._dims(tA, tB, transA, transB)
    off, total = mw.workspace_layout(plan, M, N, K)
    ws = torch.zeros(total, dtype=torch.uint8, device=dev)
    C = mw.mw_gemm(tA, tB, plan, transA=transA, transB=transB, ws=ws)
    return C.cpu().numpy(), ws, off, (M, N, K)


def narrow(plan, K):
    """The library keeps int32 diagonal sums when they cannot overflow."""
    Kp = -(-K // 64) * 64
    return min(plan.S_A, plan.S_B) * Kp * 2 ** (2 * plan.w - 2) < 2 ** 31


def partial_sums(ws, off, plan, M, N, K):
    """Partial sums as the library stores them: (D, M, N) int32 diagonal sums or
    (G, M, N) int64 group sums."""
    if narrow(plan, K):
        n = plan.D * M * N
        raw = ws[off[3]:off[3] + 4 * n].view(torch.int32).cpu().numpy().astype(np.int64)
        return raw.reshape(plan.D, N, M).transpose(0, 2, 1)       # planes are column-major
    G = -(-plan.D // plan.group)
    n = G * M * N
    raw = ws[off[3]:off[3] + 8 * n].view(torch.int64).cpu().numpy()
    return raw.reshape(G, N, M).transpose(0, 2, 1)


def oracle_partials(sp, plan, K, a, b):
    if narrow(plan, K):
        return [int(x) for x in sp.s[:, a, b]]
    bounds = [(g * plan.group, min(plan.D, (g + 1) * plan.group) - 1)
              for g in range(-(-plan.D // plan.group))]
    return slicing.group_values(sp.s[:, a, b], plan.w, bounds)


def check_ozaki(mw, cuda, A, B, plan, transA=False, transB=False, rows=None, cols=None,
                bound=True):
    C, ws, off, (M, N, K) = run(mw, cuda, A, B, plan, transA, transB)
    LA, LB = logical_pair(A, B, transA, transB)
    rows = list(range(M)) if rows is None else rows
    cols = list(range(N)) if cols is None else cols
    sp = slicing.SlicedProduct(LA, LB, plan.w, plan.S_A, plan.S_B, plan.D, rows=rows, cols=cols)
    assert sp.A.in_range and sp.B.in_range
    part = partial_sums(ws, off, plan, M, N, K)
    ref = sp.result()
    for a, i in enumerate(rows):
        for b, j in enumerate(cols):
            got = [int(part[g, i, j]) for g in range(part.shape[0])]
            assert got == oracle_partials(sp, plan, K, a, b), (i, j)
    assert np.array_equal(C[:, rows][:, :, cols], ref)
    if bound:
        ratio = exact.ExactProduct(LA, LB, rows, cols).error_ratio(C)
        assert ratio.max() <= 1.0
        return C, ratio.max()
    return C, None


@pytest.mark.parametrize("m,M,N,K,lo,hi", [
    (2, 64, 64, 64, None, None),
    (2, 130, 70, 100, -10, 10),
    (4, 40, 50, 200, -8, 8),
    (8, 33, 20, 70, None, None),
    (2, 1, 1, 1, -3, 3),
    (4, 129, 257, 65, -20, 20),
    (2, 300, 520, 100, -6, 6),      # odd number of tile rows: the last CTA pair has an empty tile
    (2, 520, 1000, 64, None, None),
    (16, 20, 24, 30, None, None),   # hexa doubles (Table 2's 16d precision)
    (16, 130, 70, 100, -3, 3),
])
def test_ozaki_bit_exact(mw, cuda, m, M, N, K, lo, hi):
    rng = SplitMix64(300 + m + M)
    if lo is None:
        A, B = uniform_mdouble(rng, m, M, K), uniform_mdouble(rng, m, K, N)
    else:
        A, B = loguniform_mdouble(rng, m, M, K, lo, hi), loguniform_mdouble(rng, m, K, N, lo, hi)
    plan = mw.plan_for(to_dev(A, cuda), to_dev(B, cuda), "ozaki")
    rows = None if M * N <= 64 * 64 else sorted(
        {i for i in (0, 1, 63, 64, 128, 255, 256, M - 2, M - 1) if 0 <= i < M})
    cols = None if M * N <= 64 * 64 else sorted(
        {j for j in (0, 5, 127, 128, 255, 256, 511, 512, N - 1) if 0 <= j < N})
    check_ozaki(mw, cuda, A, B, plan, rows=rows, cols=cols)


@pytest.mark.parametrize("transA,transB", [(True, False), (False, True), (True, True)])
def test_ozaki_transposes(mw, cuda, transA, transB):
    rng = SplitMix64(310)
    A = uniform_mdouble(rng, 2, 45, 30) if not transA else uniform_mdouble(rng, 2, 30, 45)
    B = uniform_mdouble(rng, 2, 30, 52) if not transB else uniform_mdouble(rng, 2, 52, 30)
    plan = mw.plan_for(to_dev(A, cuda), to_dev(B, cuda), "ozaki", transA, transB)
    check_ozaki(mw, cuda, A, B, plan, transA, transB)


def test_ozaki_every_diagonal_sum(mw, cuda):
    """Each stored partial sum is one diagonal sum s_t (Section 2 s_i), both when
    the library keeps them in 32 bits and, with group = 1, in 64 bits."""
    rng = SplitMix64(320)
    A, B = uniform_mdouble(rng, 2, 20, 300), uniform_mdouble(rng, 2, 300, 24)
    plan = mw.plan_for(to_dev(A, cuda), to_dev(B, cuda), "ozaki", group=1)
    C, ws, off, (M, N, K) = run(mw, cuda, A, B, plan)
    sp = slicing.SlicedProduct(A, B, plan.w, plan.S_A, plan.S_B, plan.D)
    assert np.array_equal(partial_sums(ws, off, plan, M, N, K), sp.s)
    assert np.array_equal(C, sp.result())


def test_ozaki_wide_partial_sums(mw, cuda):
    """K long enough that diagonal sums may pass 2^31: 64-bit Horner groups."""
    rng = SplitMix64(321)
    K = 9000
    A, B = uniform_mdouble(rng, 4, 40, K), uniform_mdouble(rng, 4, K, 30)
    plan = mw.plan_for(to_dev(A, cuda), to_dev(B, cuda), "ozaki")
    assert not narrow(plan, K) and plan.group > 1
    check_ozaki(mw, cuda, A, B, plan, rows=[0, 17, 39], cols=[0, 29])


@pytest.mark.parametrize("w,chunk", [(7, 1024), (7, 64), (8, 64), (6, 4096)])
def test_ozaki_other_widths_and_chunks(mw, cuda, w, chunk):
    rng = SplitMix64(330 + w)
    A, B = loguniform_mdouble(rng, 2, 70, 600, -5, 5), loguniform_mdouble(rng, 2, 600, 90, -5, 5)
    base = mw.plan_for(to_dev(A, cuda), to_dev(B, cuda), "ozaki")
    bits_a, bits_b, bits_d = base.S_A * 8, base.S_B * 8, base.D * 8
    plan = mw.mw_plan_gemm(2, "ozaki", 70, 90, 600, base.range_A, base.range_B)
    plan.w, plan.chunk = w, chunk
    plan.S_A, plan.S_B, plan.D = -(-bits_a // w), -(-bits_b // w), -(-bits_d // w)
    plan.group = 2
    check_ozaki(mw, cuda, A, B, plan, rows=[0, 33, 69], cols=[0, 44, 89])


@pytest.mark.parametrize("a,b,want", [
    # a long run of zero bits between the two words
    ([1.0, 2.0 ** -200], [1.0 + 2.0 ** -52, 3.0], [1.0 + 2.0 ** -52, 3 * 2.0 ** -200]),
    # exact tie, even mantissa kept
    ([1.0, 2.0 ** -53], [1.0, 1.0], [1.0, 2.0 ** -53]),
    # exact tie, odd mantissa rounded up, remainder negative
    ([1.0 + 2.0 ** -52, 2.0 ** -53], [1.0, 1.0], [1.0 + 2.0 ** -51, -2.0 ** -53]),
    # negative sum that one double holds exactly
    ([-1.0, 2.0 ** -53], [1.0, 1.0], [-1.0 + 2.0 ** -53]),
    # cancellation down to the last bits
    ([1.0, -1.0], [1.0 + 2.0 ** -52, 1.0], [2.0 ** -52]),
])
def test_ozaki_rounding_edge_cases(mw, cuda, a, b, want):
    """C = a . b (1 x 2 times 2 x 1, quad double): greedy words with ties to
    even and long zero runs, against the closed form and the oracle."""
    A = np.zeros((4, 1, 2)); A[0, 0, :] = a
    B = np.zeros((4, 2, 1)); B[0, :, 0] = b
    plan = mw.plan_for(to_dev(A, cuda), to_dev(B, cuda), "ozaki")
    C, _ = check_ozaki(mw, cuda, A, B, plan)
    assert list(C[:, 0, 0]) == want + [0.0] * (4 - len(want))


def test_double_double_n64_exact_check(mw, cuda):
    """Double double, n = 64, seed 0: every entry checked against the exact
    rational product, both forms."""
    A, B = dd_n64(seed=0, n=64)
    ex = exact.exact_product_full(A, B)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    for mode in ("ozaki", "plain"):
        C = mw.mw_gemm(tA, tB, mode=mode).cpu().numpy()
        worst = ex.error_ratio(C).max()
        record_worst(f"dd n=64 {mode}, all 4096 entries", worst)
        assert worst <= 1.0, mode
        for i in range(0, 64, 7):
            for j in range(0, 64, 5):
                assert exact.nonoverlapping(list(C[:, i, j])), (mode, i, j)


@pytest.mark.parametrize("m,M,N,K", [(2, 70, 90, 130), (4, 33, 40, 300), (8, 20, 17, 64)])
def test_plain_within_bound_and_close_to_fused_value(mw, cuda, m, M, N, K):
    rng = SplitMix64(340 + m)
    A, B = loguniform_mdouble(rng, m, M, K, -8, 8), loguniform_mdouble(rng, m, K, N, -8, 8)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, "plain")
    C = mw.mw_gemm(tA, tB, plan).cpu().numpy()
    rows, cols = [0, M // 2, M - 1], [0, N // 3, N - 1]
    ex = exact.ExactProduct(A, B, rows, cols)
    assert ex.error_ratio(C).max() <= 1.0
    sp = slicing.SlicedProduct(A, B, plan.w, plan.S_A, plan.S_B, plan.D, rows=rows, cols=cols)
    for a, i in enumerate(rows):
        for b, j in enumerate(cols):
            v = sp.value(a, b)               # the exact sum of the scaled diagonal sums
            err = abs(exact.to_fraction(C[:, i, j]) - v)
            assert err <= Fraction(plan.D + 2) * Fraction(2) ** (-53 * m) * ex.absum[a][b] \
                * Fraction(2) ** ex.scale


def test_zero_and_tiny_inputs(mw, cuda):
    A = np.zeros((2, 5, 7))
    B = uniform_mdouble(SplitMix64(350), 2, 7, 6)
    for mode in ("ozaki", "plain"):
        C = mw.mw_gemm(to_dev(A, cuda), to_dev(B, cuda), mode=mode).cpu().numpy()
        assert not C.any()
    # operands near the bottom of the normal range keep their scale
    A = uniform_mdouble(SplitMix64(351), 2, 6, 9) * 2.0 ** -400
    B = uniform_mdouble(SplitMix64(352), 2, 9, 5) * 2.0 ** -400
    C = mw.mw_gemm(to_dev(A, cuda), to_dev(B, cuda), mode="ozaki").cpu().numpy()
    assert exact.exact_product_full(A, B).error_ratio(C).max() <= 1.0


@pytest.mark.slow
@pytest.mark.parametrize("mode", ["ozaki", "plain"])
def test_quad_double_1024(mw, cuda, mode):
    """Quad double, M = N = K = 1024, magnitudes 2^U[-8,8), seed 1: sampled
    outputs against the exact product (and the oracle's summation for Ozaki)."""
    from synthetic import qd_1024
    A, B = qd_1024()
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, mode)
    rows, cols = [0, 1, 511, 1000, 1023], [0, 2, 640, 1023]
    if mode == "ozaki":
        _, ratio = check_ozaki(mw, cuda, A, B, plan, rows=rows, cols=cols)
    else:
        C = mw.mw_gemm(tA, tB, plan).cpu().numpy()
        ratio = exact.ExactProduct(A, B, rows, cols).error_ratio(C).max()
    record_worst(f"qd 1024^3 {mode}, 20 sampled entries", ratio)
    assert ratio <= 1.0


@pytest.mark.slow
@pytest.mark.parametrize("m", [2, 4])
def test_ozaki_4096(mw, cuda, m):
    """M = N = K = 4096, magnitudes 2^U[-20,20), seed 2: a 32 x 32 block bit for
    bit against the oracle's error-free summation (quad double: the 64-bit
    Horner partial sums of the long-K mode) and against the exact product's
    bound, plus the four corners bit for bit."""
    from synthetic import ozaki_4096
    A, B = ozaki_4096(m)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, "ozaki")
    C = mw.mw_gemm(tA, tB, plan).cpu().numpy()
    rows = cols = list(range(2048, 2080))
    worst = exact.ExactProduct(A, B, rows, cols).error_ratio(C).max()
    record_worst(f"m={m} 4096^3 ozaki, 32x32 block", worst)
    assert worst <= 1.0
    sp = slicing.SlicedProduct(A, B, plan.w, plan.S_A, plan.S_B, plan.D, rows=rows, cols=cols)
    assert np.array_equal(C[:, rows][:, :, cols], sp.result())
    r2, c2 = [0, 4095], [7, 4000]
    sp = slicing.SlicedProduct(A, B, plan.w, plan.S_A, plan.S_B, plan.D, rows=r2, cols=c2)
    assert np.array_equal(C[:, r2][:, :, c2], sp.result())


def test_stale_plan_raises(mw, cuda):
    """A plan reused on operands whose exponent spread exceeds the plan's: the
    product still runs, MW_WRANGE is raised on the GPU, and the binding turns it
    into MWRangeError by default (the bound is not guaranteed)."""
    rng = SplitMix64(370)
    A, B = loguniform_mdouble(rng, 2, 40, 50, -2, 2), loguniform_mdouble(rng, 2, 50, 30, -2, 2)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, "ozaki")
    mw.mw_gemm(tA, tB, plan)                           # fitting operands: no error
    A2 = A.copy()
    A2[:, 3, 11] *= 2.0 ** -30                         # row 3 now spans 30 more bits
    tA2 = to_dev(A2, cuda)
    with pytest.raises(mw.MWRangeError):
        mw.mw_gemm(tA2, tB, plan)
    mw.mw_gemm(tA2, tB, plan, check=False)
    assert mw.check_status(allow=mw.MW_WRANGE) == mw.MW_WRANGE
    C = mw.mw_gemm(tA2, tB, mw.plan_for(tA2, tB, "ozaki")).cpu().numpy()   # replanned
    assert exact.exact_product_full(A2, B).error_ratio(C).max() <= 1.0


def test_gemm_replays_in_a_cuda_graph(mw, cuda):
    """mw_gemm (its two operand splits forked onto a second stream and joined)
    captured in a CUDA graph: replays give the eager words, and follow new
    operand values at the same addresses."""
    rng = SplitMix64(360)
    A, B = uniform_mdouble(rng, 2, 300, 200), uniform_mdouble(rng, 2, 200, 270)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, "ozaki")
    ws = torch.empty(mw.workspace_size(plan, 300, 270, 200), dtype=torch.uint8, device=cuda)
    C = torch.empty((2, 300, 270), dtype=torch.float64, device=cuda)
    mw.mw_gemm(tA, tB, plan, C=C, ws=ws)
    torch.cuda.synchronize()
    expect = C.clone()
    C.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            mw.mw_gemm(tA, tB, plan, C=C, ws=ws, check=False)
    g.replay()
    torch.cuda.synchronize()
    mw.check_status()
    assert torch.equal(C, expect)
    tA.mul_(0.5)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(C, 0.5 * expect)
