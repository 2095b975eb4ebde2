"""mw_gemm in the residue form (MW_CRT) on the GPU against the residue oracle.

Bit for bit: the exponents, every balanced residue plane of both operands,
every int32 sum of residue products (equal to the oracle's exact sums, or
congruent to them mod p when K is long enough for the kernel to reduce), and
the final words; the words also meet the componentwise bound against the exact
product.  Sizes span several tiles with ragged tails in every dimension; the
4096^3 and 1024^3 workloads are checked on sampled blocks."""
import numpy as np
import pytest
import torch

from conftest import record_worst, to_dev
from oracle import crt, exact
from synthetic import SplitMix64, loguniform_mdouble, paper_pattern_mdouble, uniform_mdouble

pytestmark = pytest.mark.gpu


def bf16_to_int(x):
    return x.float().cpu().numpy().astype(np.int64)


def run_crt(mw, dev, A, B, plan, transA=False, transB=False):
    tA, tB = to_dev(A, dev), to_dev(B, dev)
    m, M, N, K = mw._dims(tA, tB, transA, transB)
    off, total = mw.workspace_layout(plan, M, N, K)
    ws = torch.zeros(total, dtype=torch.uint8, device=dev)
    C = mw.mw_gemm(tA, tB, plan, transA=transA, transB=transB, ws=ws)
    return C.cpu().numpy(), ws, off, (M, N, K)


def check_crt(mw, dev, A, B, plan=None, transA=False, transB=False, rows=None, cols=None,
              planes=True, label=None):
    tA, tB = to_dev(A, dev), to_dev(B, dev)
    if plan is None:
        plan = mw.plan_for(tA, tB, "crt", transA, transB)
    C, ws, off, (M, N, K) = run_crt(mw, dev, A, B, plan, transA, transB)
    rows = list(range(M)) if rows is None else rows
    cols = list(range(N)) if cols is None else cols
    moduli = mw.crt_moduli(plan.D)
    rp = crt.ResidueProduct(A, B, plan.S_A, plan.S_B, moduli, rows=rows, cols=cols,
                            transA=transA, transB=transB)
    assert rp.A.in_range and rp.B.in_range
    Kp = -(-K // 64) * 64
    D = plan.D
    ex = ws[:4 * (2 * M + 2 * N)].view(torch.int32).cpu().numpy()
    assert np.array_equal(ex[:M][rows], rp.A.E) and np.array_equal(ex[2 * M:2 * M + N][cols], rp.B.E)
    if planes:
        RA = ws[off[1]:off[1] + 2 * D * M * Kp].view(torch.bfloat16).reshape(D, M, Kp)
        RB = ws[off[2]:off[2] + 2 * D * N * Kp].view(torch.bfloat16).reshape(D, N, Kp)
        ra, rb = bf16_to_int(RA[:, rows, :K]), bf16_to_int(RB[:, cols, :K])
        assert np.array_equal(ra, rp.A.residues) and np.array_equal(rb, rp.B.residues)
        assert not bf16_to_int(RA[:, rows, K:]).any() and not bf16_to_int(RB[:, cols, K:]).any()
        # the product kernel leaves the balanced residue of every exact sum Y_p,
        # bfloat16 row-major planes [t][i][j], rows of N rounded up to 8
        ld = -(-N // 8) * 8
        R = ws[off[3]:off[3] + 2 * D * M * ld].view(torch.bfloat16).reshape(D, M, ld)[:, :, :N]
        ri = torch.tensor(rows, device=R.device)
        ci = torch.tensor(cols, device=R.device)
        R = bf16_to_int(R.index_select(1, ri).index_select(2, ci))
        for i, p in enumerate(moduli):
            h = p // 2
            assert np.array_equal(R[i], (rp.Y[i] + h) % p - h), p
    assert np.array_equal(C[:, rows][:, :, cols], rp.result())
    ratio = exact.ExactProduct(A if not transA else np.ascontiguousarray(A.transpose(0, 2, 1)),
                               B if not transB else np.ascontiguousarray(B.transpose(0, 2, 1)),
                               rows, cols).error_ratio(C).max()
    if label:
        record_worst(label, ratio)
    assert ratio <= 1.0
    return C, plan


@pytest.mark.parametrize("m,M,N,K,lo,hi", [
    (2, 64, 64, 64, None, None),
    (2, 130, 70, 100, -10, 10),       # ragged in every dimension, 128-column tiles
    (4, 40, 50, 200, -8, 8),
    (2, 1, 1, 1, -3, 3),
    (4, 129, 300, 65, -20, 20),       # 256-column tiles with a ragged second tile
    (2, 300, 520, 100, -6, 6),
    (4, 33, 20, 700, None, None),
    (4, 64, 33, 300, -45, 45),        # 81 moduli, 20 limbs of X'
    (4, 50, 40, 300, -60, 60),        # 88 moduli, 24 limbs of X'
])
def test_crt_bit_exact(mw, cuda, m, M, N, K, lo, hi):
    rng = SplitMix64(1000 + m + M + K)
    if lo is None:
        A, B = uniform_mdouble(rng, m, M, K), uniform_mdouble(rng, m, K, N)
    else:
        A, B = loguniform_mdouble(rng, m, M, K, lo, hi), loguniform_mdouble(rng, m, K, N, lo, hi)
    rows = None if M * N <= 64 * 64 else sorted(
        {i for i in (0, 1, 63, 64, 127, 128, 255, 256, M - 2, M - 1) if 0 <= i < M})
    cols = None if M * N <= 64 * 64 else sorted(
        {j for j in (0, 5, 127, 128, 255, 256, 511, 512, N - 1) if 0 <= j < N})
    check_crt(mw, cuda, A, B, rows=rows, cols=cols)


@pytest.mark.parametrize("transA,transB", [(True, False), (False, True), (True, True)])
def test_crt_transposes(mw, cuda, transA, transB):
    rng = SplitMix64(1010)
    A = uniform_mdouble(rng, 4, 45, 70) if not transA else uniform_mdouble(rng, 4, 70, 45)
    B = uniform_mdouble(rng, 4, 70, 52) if not transB else uniform_mdouble(rng, 4, 52, 70)
    check_crt(mw, cuda, A, B, transA=transA, transB=transB)


def test_crt_paper_pattern_and_zeros(mw, cuda):
    """The Section 2 bit pattern, a zero row and a zero column."""
    rng = SplitMix64(1020)
    A, B = paper_pattern_mdouble(rng, 2, 20, 96), paper_pattern_mdouble(rng, 2, 96, 18)
    A[:, 3, :] = 0.0
    B[:, :, 5] = 0.0
    C, _ = check_crt(mw, cuda, A, B)
    assert not C[:, 3, :].any() and not C[:, :, 5].any()


@pytest.mark.parametrize("m,M,N,K,lead", [(4, 70, 45, 130, False), (2, 2048, 2048, 2048, True)])
def test_crt_entries_not_normalised(mw, cuda, m, M, N, K, lead):
    """Entries whose later word is larger than the first (a zero leading word, a
    last word far above the first) in rows of A and a column of B.  Operands of
    at least 2^22 entries take the exponents from the leading words and the
    residue split checks every entry: such an operand is cut again with the
    exponents over every word (the flags after the largest spreads say which).
    Either way the exponents, residues and words equal the oracle's bit for bit."""
    rng = SplitMix64(1025 + m)
    A, B = uniform_mdouble(rng, m, M, K), uniform_mdouble(rng, m, K, N)

    def flags(ws):
        return ws[4 * (2 * M + 2 * N + 2):4 * (2 * M + 2 * N + 4)].view(torch.int32).cpu().tolist()

    _, ws, _, _ = run_crt(mw, cuda, A, B, mw.plan_for(to_dev(A, cuda), to_dev(B, cuda), "crt"))
    assert flags(ws) == [0, 0]
    A[0, 3, 5] = 0.0
    A[1, 3, 5] = 2.0                      # row 3: leading word zero, second word 2
    A[0, 1, 0] = 1e-3
    A[m - 1, 1, 0] = 4.0                  # row 1: the last word far above the first
    B[0, 2, 4] = 0.0
    B[m - 1, 2, 4] = -8.0                 # column 4 of B
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, "crt")
    rows = None if not lead else [0, 1, 3, 1000, M - 1]
    cols = None if not lead else [0, 4, 777, N - 1]
    check_crt(mw, cuda, A, B, plan=plan, rows=rows, cols=cols)
    _, ws, _, _ = run_crt(mw, cuda, A, B, plan)
    assert flags(ws) == ([1, 1] if lead else [0, 0])
    mw.check_status()


def test_crt_long_k_reduces_mod_p(mw, cuda):
    """K = 40,000 quad doubles: the moduli above 363 drain every 64 products and
    reduce their int32 sums mod p every 511 drains; the stored residues equal
    those of the oracle's exact sums and the words stay bit-exact."""
    rng = SplitMix64(1030)
    K = 40000
    A, B = loguniform_mdouble(rng, 4, 3, K, -4, 4), loguniform_mdouble(rng, 4, K, 3, -4, 4)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, "crt")
    plan.D = max(plan.D, 75)          # more moduli than needed, up to some above 363
    assert any(p > 363 for p in mw.crt_moduli(plan.D))
    check_crt(mw, cuda, A, B, plan=plan)


def test_crt_matches_the_slice_form_with_every_pair(mw, cuda):
    """With L = 8 S the residue form and the slice form keeping every pair give
    the same words (the same exact integer, rounded the same way)."""
    rng = SplitMix64(1040)
    A, B = loguniform_mdouble(rng, 2, 70, 90, -6, 6), loguniform_mdouble(rng, 2, 90, 60, -6, 6)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    po = mw.plan_for(tA, tB, "ozaki")
    po.D = po.S_A + po.S_B - 1
    pc = mw.plan_for(tA, tB, "crt")
    pc.S_A, pc.S_B = 8 * po.S_A, 8 * po.S_B
    ps = mw.crt_moduli()
    need = 8 * 90 * 2 ** (pc.S_A + pc.S_B - 2)
    pc.D = next(n for n in range(1, len(ps) + 1) if crt.modulus_product(ps[:n]) > need)
    Co = mw.mw_gemm(tA, tB, po)
    Cc = mw.mw_gemm(tA, tB, pc)
    assert torch.equal(Co, Cc)


def test_crt_replays_in_a_cuda_graph(mw, cuda):
    rng = SplitMix64(1050)
    A, B = uniform_mdouble(rng, 2, 300, 200), uniform_mdouble(rng, 2, 200, 270)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, "crt")
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


def test_crt_status_bits(mw, cuda):
    """Non-finite input raises MW_ENONFINITE, an entry whose second word is far
    above its first (not normalised) raises MW_ERANGE, a clean call nothing."""
    rng = SplitMix64(1060)
    A, B = uniform_mdouble(rng, 2, 10, 30), uniform_mdouble(rng, 2, 30, 12)
    tA, tB = to_dev(A, cuda), to_dev(B, cuda)
    plan = mw.plan_for(tA, tB, "crt")
    mw.get_status(clear=True)
    A2 = A.copy()
    A2[1, 2, 3] = np.inf
    mw.mw_gemm(to_dev(A2, cuda), tB, plan, check=False)
    assert mw.get_status(clear=True) & mw.MW_ENONFINITE
    A3 = A.copy()
    A3[1, 4, 6] = A3[0, 4, 6] * 2.0 ** 200    # far above the row's shared exponent
    A3[0, 4, 6] = 2.0 ** -900
    mw.mw_gemm(to_dev(A3, cuda), tB, plan, check=False)
    assert mw.get_status(clear=True) & (mw.MW_ERANGE | mw.MW_WRANGE)
    mw.mw_gemm(tA, tB, plan)
    assert mw.get_status(clear=True) == 0


@pytest.mark.slow
def test_crt_quad_double_1024(mw, cuda):
    from synthetic import qd_1024
    A, B = qd_1024()
    check_crt(mw, cuda, A, B, rows=[0, 1, 511, 1000, 1023], cols=[0, 2, 640, 1023],
              label="qd 1024^3 crt, 20 sampled entries")


@pytest.mark.slow
@pytest.mark.parametrize("m", [2, 4])
def test_crt_4096(mw, cuda, m):
    """M = N = K = 4096, magnitudes 2^U[-20,20), seed 2 (the benchmark's operands):
    for a 32 x 32 block, the exponents, every residue plane of its 32 rows of op(A)
    and 32 columns of op(B) (the leading-word exponent pass of operands this
    large), the product kernel's residue of every sum and the words bit for bit
    against the residue oracle and within the bound; the corners bit for bit."""
    from synthetic import ozaki_4096
    A, B = ozaki_4096(m)
    rows = cols = list(range(2048, 2080))
    C, plan = check_crt(mw, cuda, A, B, rows=rows, cols=cols,
                        label=f"m={m} 4096^3 crt, 32x32 block")
    rp = crt.ResidueProduct(A, B, plan.S_A, plan.S_B, mw.crt_moduli(plan.D), rows=[0, 4095],
                            cols=[7, 4000])
    assert np.array_equal(C[:, [0, 4095]][:, :, [7, 4000]], rp.result())
