"""mw_gemm_batched: every problem of a batch equals the single product with the
same plan bit for bit, and sampled problems equal the oracle's error-free
summation bit for bit and meet the bound against the exact product."""
import numpy as np
import pytest
import torch

from conftest import record_worst, to_dev
from oracle import exact, slicing
from synthetic import SplitMix64, batch_flat, batch_sizes, loguniform_mdouble, uniform_mdouble

pytestmark = pytest.mark.gpu


def single(mw, A, B, plan):
    return mw.mw_gemm(A, B, plan)


@pytest.mark.parametrize("m", [2, 4, 8, 16])
def test_batch_of_uneven_products(mw, cuda, m):
    rng = SplitMix64(600 + m)
    shapes = [(1, 1, 1), (8, 8, 8), (130, 7, 64), (17, 200, 65), (128, 128, 128), (3, 129, 300),
              (64, 33, 9), (257, 40, 31)]
    As = [to_dev(loguniform_mdouble(rng, m, M, K, -6, 6), cuda) for M, N, K in shapes]
    Bs = [to_dev(loguniform_mdouble(rng, m, K, N, -6, 6), cuda) for M, N, K in shapes]
    batch = mw.Batch(As, Bs)
    Cs = batch.run()
    mw.check_status()
    plan = batch.plan_
    for i, (A, B, C) in enumerate(zip(As, Bs, Cs)):
        ref = single(mw, A, B, plan)
        assert torch.equal(C, ref), i
    # two problems against the oracle, bit for bit and within the bound
    for i in (2, 4):
        An, Bn = As[i].cpu().numpy(), Bs[i].cpu().numpy()
        M, N = An.shape[1], Bn.shape[2]
        rows, cols = [0, M // 2, M - 1], [0, N - 1]
        sp = slicing.SlicedProduct(An, Bn, plan.w, plan.S_A, plan.S_B, plan.D, rows=rows, cols=cols)
        C = Cs[i].cpu().numpy()
        assert np.array_equal(C[:, rows][:, :, cols], sp.result())
        assert exact.ExactProduct(An, Bn, rows, cols).error_ratio(C).max() <= 1.0


def test_batch_entries_not_normalised(mw, cuda):
    """Octo doubles whose later word is larger than the first, in a row of A and
    a column of B: the splits take the exponents from the leading words, find
    the larger word while cutting and cut that row or stripe again; every
    problem still equals the single product and the oracle bit for bit."""
    m = 8
    rng = SplitMix64(620)
    shapes = [(40, 50, 30), (70, 9, 100), (9, 70, 64)]
    As, Bs = [], []
    for M, N, K in shapes:
        A = uniform_mdouble(rng, m, M, K)
        B = uniform_mdouble(rng, m, K, N)
        A[0, 3, 5] = 0.0
        A[1, 3, 5] = 2.0                  # row 3: leading word zero, second word 2
        A[0, 1, 0] = 1e-3
        A[m - 1, 1, 0] = 4.0              # row 1: the last word far above the first
        B[0, 2, 4] = 0.0
        B[2, 2, 4] = -8.0                 # column 4 of B
        As.append(to_dev(A, cuda))
        Bs.append(to_dev(B, cuda))
    batch = mw.Batch(As, Bs)
    Cs = batch.run()
    mw.check_status()
    plan = batch.plan_
    for i, (A, B, C) in enumerate(zip(As, Bs, Cs)):
        assert torch.equal(C, single(mw, A, B, plan)), i
        An, Bn = A.cpu().numpy(), B.cpu().numpy()
        M, N = An.shape[1], Bn.shape[2]
        rows, cols = sorted({0, 1, 3, M - 1}), sorted({0, 4, N - 1})
        sp = slicing.SlicedProduct(An, Bn, plan.w, plan.S_A, plan.S_B, plan.D, rows=rows, cols=cols)
        assert sp.A.in_range and sp.B.in_range
        assert np.array_equal(C.cpu().numpy()[:, rows][:, :, cols], sp.result()), i


def test_packed_batch_equals_list_batch(mw, cuda):
    """Batch.packed (descriptors from flat tensors, no per-problem loop) gives
    the same words as the list form, with rectangular problems at offsets."""
    rng = SplitMix64(605)
    shapes = [(5, 7, 3), (64, 1, 130), (40, 33, 64), (1, 90, 17)]
    m = 4
    oA, oB, oC = [], [], []
    a = b = c = 0
    for M, N, K in shapes:
        oA.append(a); oB.append(b); oC.append(c)
        a += M * K + 3; b += K * N + 5; c += M * N + 1      # gaps between problems
    FA = uniform_mdouble(rng, m, 1, a)[:, 0, :]
    FB = uniform_mdouble(rng, m, 1, b)[:, 0, :]
    dA, dB = to_dev(np.ascontiguousarray(FA), cuda), to_dev(np.ascontiguousarray(FB), cuda)
    dC = torch.zeros((m, c), dtype=torch.float64, device=cuda)
    As = [dA[:, o:o + M * K].view(m, M, K) for o, (M, N, K) in zip(oA, shapes)]
    Bs = [dB[:, o:o + K * N].view(m, K, N) for o, (M, N, K) in zip(oB, shapes)]
    ref = mw.Batch(As, Bs)
    ref.run()
    packed = mw.Batch.packed(dA, dB, dC, shapes, list(zip(oA, oB, oC)), plan=ref.plan_)
    packed.run()
    mw.check_status()
    for o, (M, N, K), C in zip(oC, shapes, ref.Cs):
        assert torch.equal(dC[:, o:o + M * N].view(m, M, N), C)
    with pytest.raises(mw.MWError):
        mw.Batch.packed(dA, dB, dC, [(5, 7, 3)], [(a, 0, 0)])       # outside A


def test_batch_replays_in_a_cuda_graph(mw, cuda):
    rng = SplitMix64(610)
    sizes = [40, 9, 77, 128, 16]
    As = [to_dev(uniform_mdouble(rng, 2, n, n), cuda) for n in sizes]
    Bs = [to_dev(uniform_mdouble(rng, 2, n, n), cuda) for n in sizes]
    batch = mw.Batch(As, Bs)
    batch.run()                                   # first call outside the capture
    torch.cuda.synchronize()
    expect = [c.clone() for c in batch.Cs]
    for c in batch.Cs:
        c.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.run()
    g.replay()
    torch.cuda.synchronize()
    mw.check_status()
    for c, e in zip(batch.Cs, expect):
        assert torch.equal(c, e)
    # new operand values at the same addresses: the replay follows them
    for a in As:
        a.mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    for c, e in zip(batch.Cs, expect):
        assert torch.equal(c, 2.0 * e)


@pytest.mark.slow
def test_octo_double_batch_20000(mw, cuda):
    """20,000 octo-double products, n ~ U{8..128}, seed 3: every problem against
    the single product bit for bit, a seeded sample of 200 against the oracle."""
    sizes = batch_sizes(20000, 8, 128, seed=3)
    FA, FB, offs = batch_flat(sizes, m=8, seed=3)
    dA, dB = to_dev(FA, cuda), to_dev(FB, cuda)
    As, Bs = [], []
    for n, o in zip(sizes, offs):
        n, o = int(n), int(o)
        As.append(dA[:, o:o + n * n].view(8, n, n))
        Bs.append(dB[:, o:o + n * n].view(8, n, n))
    order = np.argsort(-sizes, kind="stable")       # largest first
    batch = mw.Batch([As[i] for i in order], [Bs[i] for i in order])
    batch.run()
    mw.check_status()
    Cs = [None] * len(sizes)
    for k, i in enumerate(order):
        Cs[i] = batch.Cs[k]
    plan = batch.plan_
    for i in range(len(sizes)):
        assert torch.equal(Cs[i], mw.mw_gemm(As[i], Bs[i], plan, check=False)), i
    mw.check_status()
    rng = SplitMix64(620)
    sample = [int(x) for x in rng.next(200) % np.uint64(len(sizes))]
    worst = 0.0
    for i in sample:
        An, Bn, C = As[i].cpu().numpy(), Bs[i].cpu().numpy(), Cs[i].cpu().numpy()
        n = An.shape[1]
        rows, cols = [0, n - 1], [n // 2]
        sp = slicing.SlicedProduct(An, Bn, plan.w, plan.S_A, plan.S_B, plan.D, rows=rows, cols=cols)
        assert np.array_equal(C[:, rows][:, :, cols], sp.result()), i
        worst = max(worst, exact.ExactProduct(An, Bn, rows, cols).error_ratio(C).max())
    record_worst("20,000 od products, 200 sampled problems x 2 entries", worst)
    assert worst <= 1.0


def test_batch_wide_partial_sums(mw, cuda):
    """A batch whose longest K makes diagonal sums pass 2^31: 64-bit Horner
    groups on 128 x 128 tiles, one B slice per MMA; every problem equals the
    single product bit for bit, two entries the oracle."""
    rng = SplitMix64(640)
    shapes = [(20, 30, 9000), (5, 7, 100), (130, 9, 2500)]
    As = [to_dev(uniform_mdouble(rng, 2, M, K), cuda) for M, N, K in shapes]
    Bs = [to_dev(uniform_mdouble(rng, 2, K, N), cuda) for M, N, K in shapes]
    batch = mw.Batch(As, Bs)
    plan = batch.plan_
    Kp = -(-9000 // 64) * 64
    assert min(plan.S_A, plan.S_B) * Kp * 2 ** (2 * plan.w - 2) >= 2 ** 31   # wide
    Cs = batch.run()
    mw.check_status()
    for A, B, C in zip(As, Bs, Cs):
        assert torch.equal(C, mw.mw_gemm(A, B, plan))
    An, Bn = As[0].cpu().numpy(), Bs[0].cpu().numpy()
    sp = slicing.SlicedProduct(An, Bn, plan.w, plan.S_A, plan.S_B, plan.D, rows=[0, 19], cols=[29])
    assert np.array_equal(Cs[0].cpu().numpy()[:, [0, 19]][:, :, [29]], sp.result())
