#!/usr/bin/env python
"""Benchmark of the m-double matrix product on GB300.

Default workload (the benchmark line): M = N = K = 4096, quad double and
double double, every leading word of magnitude 2^U[-20, 20) with a random sign
and lower words scaled by 2^-53 U[-1,1) (seed 2).  One step is the whole
product through the C interface: exponents and pieces of both operands, the
tensor-core products of pieces with their exact integer drains, and the exact
fusion into m words (the Ozaki form).  `value` is the quad-double step; the
double-double step, the plain FP64 form of the paper (MW_PLAIN) on the same
operands and error bound, and the quad-double 1024^3 product are sub-records of
the same line.

Printed: one JSON line (rank 0).  value = m-double GFLOP/s = 2 M N K / time,
summed over ranks (each rank a replica).  L2 is flushed (a 256 MiB write)
before every timed step; steps are timed with CUDA events on the stream the
library launches on.  `--impl reference` times the CPU oracle (textbook
m-double product, all host cores) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "m-double GEMM GFLOP/s (dd,qd) Ozaki-INT8 vs FP64 plain, same error bound"
HEADLINE = ("m-double GEMM C=A*B, M=N=K=4096, quad double (value) and double double, leading "
            "words 2^U[-20,20) random sign, lower words x2^-53 U[-1,1), seed 2; Ozaki form next "
            "to the plain FP64 form at the same error bound")
KERNELS_PER_STEP = 8   # per operand: exponent, finalize, pieces (x2); product; combine
LEAD_MIN_ENTRIES = 1 << 22   # residue form: operands this large take leading-word exponents


def kernels_per_step(mode, M, N, K):
    """The library's kernel launches in one product: per operand exponents,
    finalize and pieces (the residue form's large operands: leading-word
    exponents, finalize, residues, then the pass over every word, finalize and
    residues again, which return at once when not needed); product; combine."""
    if mode != "crt":
        return KERNELS_PER_STEP
    return sum(6 if R * K >= LEAD_MIN_ENTRIES else 3 for R in (M, N)) + 2
WORD_NAMES = {2: "double double", 4: "quad double", 8: "octo double", 16: "hexa double"}


def dtype_of(m, pieces="exact integer slices; bf16 operands on tcgen05"):
    """The arithmetic the path computes in: an m-double result built from exact
    integer pieces (not a reduced-precision result)."""
    return f"f64x{m} ({WORD_NAMES[m]} result; {pieces})"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mw", choices=["mw", "reference"])
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="timed runs of the plain FP64 form (0 = leave it out)")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="end-to-end runs from host memory (-1 = steps/4, at least 3; 0 = leave out)")
    ap.add_argument("--cpu-seconds", type=float, default=8.0,
                    help="target seconds of each CPU oracle sample (0 = leave the CPU leg out)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-graph", action="store_true",
                    help="single products: launch each step directly instead of replaying a graph")
    ap.add_argument("--forms", default="ozaki,crt", type=lambda s: s.split(","),
                    help="headline: Ozaki forms to time (ozaki = digit slices, crt = residues)")
    ap.add_argument("--mode", default="crt", choices=["ozaki", "crt", "textbook"],
                    help="single workloads: the form to time")
    ap.add_argument("--size", type=int, default=0,
                    help="single workloads: M = N = K (0 = the workload's own size; smaller "
                         "sizes of the same recipe are for profiling)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="headline: leave out the autotuner's timing of every admissible plan")
    ap.add_argument("--no-secondary", action="store_true",
                    help="headline: leave out the quad-double 1024^3 sub-record")
    ap.add_argument("--m", type=int, default=4, choices=[2, 4, 8, 16],
                    help="table2, elementwise: words per m-double (2, 4, 8 or 16; elementwise 2-8)")
    ap.add_argument("--op", default="div", choices=["add", "mul", "div"],
                    help="elementwise: the m-double operation (Table 1's add, mul, div)")
    ap.add_argument("--count", type=int, default=20000,
                    help="od_batch: number of products (20,000 is the benchmark; fewer for profiling)")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "qd1024", "dd4096", "qd4096", "od_batch", "adjoint",
                             "table2", "series", "elementwise"],
                    help="headline (default): the benchmark line, quad and double double at "
                         "4096^3; the others measure one configuration of the method each")
    return ap.parse_args()


def dist_setup(n):
    import torch
    import torch.distributed as dist
    if n > 1 or "WORLD_SIZE" in os.environ and int(os.environ.get("WORLD_SIZE", "1")) > 1:
        dist.init_process_group("nccl")
        rank = dist.get_rank()
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
        return dist, rank, dist.get_world_size()
    return None, 0, 1


def aggregate(t_local_s: float, flops_per_step: float, steps: int, dist=None, device=None):
    """Whole-job throughput of N replicas: every rank did the same work, the job
    took as long as the slowest rank.  Returns (value GFLOP/s, max time s)."""
    t = t_local_s
    world = 1
    if dist is not None:
        import torch
        world = dist.get_world_size()
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return world * flops_per_step * steps / t / 1e9, t


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("bf16_tflops"), d.get("bf16_tflops_sustained"), d.get("hbm_gbs"), "measured"
    return 1900.0, 1700.0, 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_sample(A, B, target_s, label):
    """The oracle's textbook m-double product on a bounded sample of C: a block
    of rows (spread over A) times the first columns of B, sized from a short
    single-thread calibration so that the sample takes about target_s seconds
    on all host cores.  Returns the cpu_baseline record."""
    from oracle import textbook
    tc = textbook.TextbookC()
    threads = tc.max_threads()
    m, M, K = A.shape
    N = B.shape[2]
    cols = min(N, 256)
    Bs = np.ascontiguousarray(B[:, :, :cols])
    t0 = time.perf_counter()
    tc.gemm(A, Bs, rows=[0], threads=1)
    one = max(time.perf_counter() - t0, 1e-6)            # one row of `cols` outputs
    rows = int(max(threads, min(M, target_s * threads / one)))
    if rows >= M and cols < N:                            # the whole block is cheap: widen it
        cols = int(min(N, cols * max(1.0, target_s * threads / (one * M))))
        Bs = np.ascontiguousarray(B[:, :, :cols])
        rows = M
    sel = np.linspace(0, M - 1, rows).astype(np.int64)
    t0 = time.perf_counter()
    tc.gemm(A, Bs, rows=sel, threads=threads)
    dt = time.perf_counter() - t0
    flops = 2.0 * rows * cols * K
    return {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"{rows} rows x {cols} columns of the {M}x{N} C ({label}, every output a "
                      f"full K = {K} inner product), {dt:.2f} s"}


def run_reference(args):
    """The oracle's textbook product on the benchmark line's workload (quad
    double 4096^3), every step a bounded sample of it on all host cores."""
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and int(os.environ.get("RANK", "0")) != 0:
        return
    import synthetic
    A, B = synthetic.ozaki_4096(4)
    per_step = max(1.0, 90.0 / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        cpu_sample(A, B, per_step / 4, "warm-up")
    vals = [cpu_sample(A, B, per_step, "quad double") for _ in range(args.steps)]
    value = statistics.mean(v["value"] for v in vals)
    ms = 2.0 * 4096 ** 3 / (value * 1e9) * 1e3                  # one whole product
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64x4 (quad double result; textbook two-sum and "
                                          "Dekker two-product on the host)",
            "data": "synthetic",
            "config": {"workload": HEADLINE, "m": 4, "M": 4096, "N": 4096, "K": 4096,
                       "form": "textbook m-double (two-sum, Dekker two-product), CPU oracle",
                       "ms_per_step_is": "one whole 4096^3 product at the sampled rate"},
            "cpu_baseline": vals[-1],
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


WORKLOADS = {
    # name: (m, n, generator, description)
    "qd1024": (4, 1024, "qd_1024", "quad-double GEMM C=A*B, M=N=K=1024, leading words "
               "2^U[-8,8) random sign, lower words x2^-53 U[-1,1), seed 1"),
    "dd4096": (2, 4096, "ozaki_4096", "double-double GEMM M=N=K=4096, leading words 2^U[-20,20) "
               "random sign, lower words x2^-53 U[-1,1), seed 2"),
    "qd4096": (4, 4096, "ozaki_4096", "quad-double GEMM M=N=K=4096, leading words 2^U[-20,20) "
               "random sign, lower words x2^-53 U[-1,1), seed 2"),
}


def single_inputs(name, size=0):
    import synthetic
    m, n, gen, _ = WORKLOADS[name]
    n = size or n
    if gen == "qd_1024":
        return synthetic.qd_1024(seed=1, n=n)
    return synthetic.ozaki_4096(m, seed=2, n=n)


def timed(step, steps, flush, mw, dist, dev, phase=True):
    """Run `steps` steps with an untimed L2 flush before each; CUDA events on the
    current stream; returns (per-step ms, product-kernel ms, clocks) and, with
    phase events, leaves the mean ms of the split, product and fusion phases in
    timed.phases."""
    import torch
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    clocks = Clocks(dev.index)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for s in range(steps):
        flush.fill_(float(s))
        if phase:
            mw.set_phase_events(ev[s])
        else:
            ev[s][0].record()
        step()
        if not phase:
            ev[s][3].record()
    mw.set_phase_events(None)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    mw.check_status()
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    kern_ms = [e[1].elapsed_time(e[2]) for e in ev] if phase else []
    timed.phases = ({"split_ms": statistics.mean(e[0].elapsed_time(e[1]) for e in ev),
                     "product_ms": statistics.mean(kern_ms),
                     "fusion_ms": statistics.mean(e[2].elapsed_time(e[3]) for e in ev)}
                    if phase else None)
    return step_ms, kern_ms, clk


# DRAM bytes (read + write) of one product-kernel launch, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum), with the digest of the
# kernel's sources at capture time: a changed kernel reports no traffic until it
# is captured again.
KERNEL_SOURCES = ("mw_ozaki.cu", "mw_tc.cuh", "mw_device.cuh", "mw_work.cuh")
TRAFFIC = {
    "qd1024": {"bytes": 394153216 + 85361664, "digest": "9ce880bc15265ecb"},
    # 2,000 of the 20,000 products captured (the whole batch holds ~100 GB), x10
    "od_batch": {"bytes": 10 * (2874157056 + 2759791616), "digest": "9ce880bc15265ecb"},
    # residue form, captured at 2048^3 (quad double 64 moduli, double double 37) and
    # scaled by 4: residue planes in and residues out both grow with N^2
    "qd4096_crt": {"bytes": 4 * (1073851648 + 508689920), "digest": "9ce880bc15265ecb"},
    "dd4096_crt": {"bytes": 4 * (620855040 + 281017600), "digest": "9ce880bc15265ecb"},
}


def kernel_digest():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2606_20863_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def workload_key(m, M, N, K, mode="ozaki"):
    """Name of a captured single-product workload, for its DRAM traffic."""
    base = {(4, 1024): "qd1024", (2, 4096): "dd4096", (4, 4096): "qd4096"}.get(
        (m, M), None) if M == N == K else None
    return None if base is None else (base if mode == "ozaki" else f"{base}_{mode}")


def traffic_of(workload):
    t = TRAFFIC.get(workload)
    return t["bytes"] if t and t["digest"] == kernel_digest() else None


def roofline_of(pairs, flops_per_pair, kern_ms, workload=None):
    bf16_burst, _, _, peak_src = load_peaks()
    kern_s = statistics.mean(kern_ms) / 1e3
    achieved = pairs * flops_per_pair / kern_s / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": bf16_burst, "unit": "TFLOP/s",
            "frac": achieved / bf16_burst, "traffic": traffic_of(workload),
            "kernel": "ozaki_kernel (tcgen05 kind::f16, bf16 integer slices or residues)",
            "peak_source": f"{peak_src} bf16 dense burst (MEASURED_PEAKS.json)",
            "algorithmic": f"{pairs} tensor-core products (slice pairs or moduli) x "
                           f"{flops_per_pair:.4g} flop = {pairs * flops_per_pair:.3e} flop "
                           "per launch"}


TABLE1_MUL_ADD = {2: 43, 4: 425, 8: 2011}   # Table 1: double ops of one m-double add + mul


def measure_pipes(torch, dev):
    """FP64 and INT8 throughput of this GPU through the library GEMMs of torch
    (cuBLAS): the denominators of the plain form and the INT8 context."""
    def best(f, flops, n=3):
        f(); torch.cuda.synchronize()
        t = []
        for _ in range(n):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(); f(); b.record(); b.synchronize()
            t.append(a.elapsed_time(b) / 1e3)
        return flops / min(t) / 1e12
    n = 4096
    x = torch.randn(n, n, dtype=torch.float64, device=dev)
    fp64 = best(lambda: x @ x, 2.0 * n ** 3)
    del x
    xi = torch.randint(-128, 127, (n, n), dtype=torch.int8, device=dev)
    yi = torch.randint(-128, 127, (n, n), dtype=torch.int8, device=dev).t().contiguous().t()
    try:
        int8 = best(lambda: torch._int_mm(xi, yi), 2.0 * n ** 3)
    except Exception:
        int8 = None
    return fp64, int8


def count_pairs(plan):
    """Tensor-core products of one launch: kept slice pairs, or one per modulus
    in the residue form."""
    if plan.mode == 3:                                   # MW_CRT
        return plan.D
    return sum(1 for t in range(plan.D) for p in range(plan.S_A) if 0 <= t - p < plan.S_B)


FORMS = {"textbook": "textbook ('ordinary') m-double product on the FP64 pipe: two_prod, "
                     "two_sum and m-word renormalisation per term, k in order",
         "ozaki": "Ozaki slices: bf16 integer digits on tcgen05, every kept pair of digit "
                  "matrices, fp32 drained to integers, exact fusion",
         "crt": "Ozaki residues (scheme II): balanced residues modulo pairwise coprime moduli "
                "on tcgen05, one product per modulus, Chinese-remainder reconstruction"}


def e2e_pipelined(torch, steps, h_in, compute):
    """End to end through the public call, as a stream of steps would run:
    step i's pinned host inputs are copied in on one stream and its results
    copied out to pinned host buffers on another while the GPU computes the
    step before or after it (two device buffers of each input, ordered by
    events).  Every step's copies and its call lie inside the timed region.
    compute(device inputs) -> list of device outputs.  Two untimed steps first
    (one per buffer, so that no allocation falls in the timed steps); returns
    seconds per timed step."""
    cur = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    d_in = [[torch.empty(h.shape, dtype=h.dtype, device=cur.device) for h in h_in] for _ in range(2)]
    ev_in, ev_comp, ev_out = ([torch.cuda.Event() for _ in range(2)] for _ in range(3))
    h_out = [None, None]
    used = [False, False]
    t0 = None
    for i in range(steps + 2):
        if i == 2:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        k = i % 2
        with torch.cuda.stream(s_in):
            if used[k]:
                s_in.wait_event(ev_comp[k])          # step i-2 has read this buffer
            for d, h in zip(d_in[k], h_in):
                d.copy_(h, non_blocking=True)
            ev_in[k].record(s_in)
        cur.wait_event(ev_in[k])
        outs = compute(d_in[k])
        ev_comp[k].record(cur)
        if h_out[0] is None:                          # pinned buffers before the timed steps
            h_out = [[torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs]
                     for _ in range(2)]
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[k])
            for h, o in zip(h_out[k], outs):
                o.record_stream(s_out)
                h.copy_(o, non_blocking=True)
            ev_out[k].record(s_out)
        used[k] = True
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / steps


E2E_HOW = ("pinned host inputs copied in and results copied out every step, on two copy "
           "streams overlapping the neighbouring steps' compute (two steps in flight)")


def measure_single(args, mw, torch, dist, rank, dev, A, B, workload, mode="ozaki",
                   graph=False, plain_steps=0, e2e_steps=0, cpu_s=0.0, pipes=None):
    """One single-product workload in one form: the step (`steps` timed runs,
    L2 flushed before each), its product-kernel time from phase events around
    direct calls, optionally the plain FP64 form on the same operands (same
    error bound), the end-to-end rate through the public call from pinned host
    buffers (one plan made before the loop, as a caller with fixed-range
    operands would), and the CPU oracle on a bounded sample.  Returns a record
    with the device-timed value aggregated over ranks."""
    m, M, K = A.shape
    N = B.shape[2]
    tA = torch.from_numpy(A).to(dev)
    tB = torch.from_numpy(B).to(dev)
    flops = 2.0 * M * N * K
    plan = mw.plan_for(tA, tB, mode)
    ws = torch.empty(mw.workspace_size(plan, M, N, K), dtype=torch.uint8, device=dev)
    C = torch.empty((m, M, N), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pairs = count_pairs(plan) if mode != "textbook" else 0

    def call():
        mw.mw_gemm(tA, tB, plan, C=C, ws=ws, check=False)

    call()
    torch.cuda.synchronize()
    mw.check_status()
    g = None
    if graph:
        # one product call captured in a CUDA graph and replayed per step (the
        # launches of the splits, product and fusion without host gaps)
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream()
        with torch.cuda.stream(gs):
            with torch.cuda.graph(g, stream=gs):
                call()
    step = g.replay if g is not None else call
    for _ in range(args.warmup):
        step()
    mw.check_status()
    torch.cuda.synchronize()
    step_ms, _, clk = timed(step, args.steps, flush, mw, dist, dev, phase=False)
    value, t_step = aggregate(sum(step_ms) / 1e3, flops, args.steps, dist, dev)
    # product-kernel time: phase events around direct calls (events are not
    # recorded inside a graph), as many runs as timed steps
    _, kern_ms, _ = timed(call, args.steps, flush, mw, None, dev)
    phases = timed.phases
    rec = {"workload": workload, "mode": mode, "m": m, "M": M, "N": N, "K": K, "value": value,
           "unit": "GFLOP/s", "ms_per_step": t_step * 1e3 / args.steps,
           "step_ms_min": min(step_ms), "product_kernel_ms": statistics.mean(kern_ms),
           "phases_ms_direct_calls": phases, "plan": plan.as_dict(),
           "tensor_products_per_launch": pairs, "form": FORMS[mode],
           "launch": "one mw_gemm call captured in a CUDA graph, replayed per step"
                     if g is not None else "direct mw_gemm calls",
           "roofline": roofline_of(pairs, flops, kern_ms, workload_key(m, M, N, K, mode))
                       if mode != "textbook" else None,
           "clocks": clk, "gpu_launches": kernels_per_step(mode, M, N, K) * args.steps}
    del g
    extras(args, mw, torch, dist, rank, dev, A, B, tA, tB, plan, rec, plain_steps, e2e_steps,
           cpu_s, pipes)
    del tA, tB, ws, C, flush
    torch.cuda.empty_cache()
    return rec


def extras(args, mw, torch, dist, rank, dev, A, B, tA, tB, plan, rec, plain_steps, e2e_steps,
           cpu_s, pipes):
    """The plain FP64 form, the end-to-end rate and the CPU oracle for a record."""
    m, M, K = A.shape
    N = B.shape[2]
    flops = 2.0 * M * N * K
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # plain FP64 form on the same operands and bound (the comparison of the metric)
    if plain_steps > 0:
        pplan = mw.plan_for(tA, tB, "plain")
        pws = torch.empty(mw.workspace_size(pplan, M, N, K), dtype=torch.uint8, device=dev)
        Cp = torch.empty((m, M, N), dtype=torch.float64, device=dev)
        if M * N * K <= 1024 ** 3:                 # one untimed call (4096^3 takes seconds)
            mw.mw_gemm(tA, tB, pplan, C=Cp, ws=pws)
        pms, _, pclk = timed(lambda: mw.mw_gemm(tA, tB, pplan, C=Cp, ws=pws, check=False),
                             plain_steps, flush, mw, None, dev, phase=False)
        plain = flops * plain_steps / (sum(pms) / 1e3) / 1e9
        rec["plain"] = {"value": plain, "unit": "GFLOP/s", "steps": plain_steps,
                        "ms_per_step": sum(pms) / plain_steps, "plan": pplan.as_dict(),
                        "form": "MW_PLAIN: double pieces, FP64 FMA, m-double fusion",
                        "clocks": pclk}
        if pipes:
            fp64_peak = pipes[0]
            ppairs = count_pairs(pplan)
            roof = 2.0 * fp64_peak * 1e3 / TABLE1_MUL_ADD[m]     # m-double GFLOP/s
            rec["plain"]["roofline"] = {
                "bound": "fp64", "peak_from_table1_gflops": roof,
                "frac_of_table1_roofline": plain / roof,
                "fp64_pipe_tflops": ppairs * plain / 1e3,
                "fp64_pipe_frac": ppairs * plain / 1e3 / fp64_peak,
                "fp64_peak_tflops_measured": fp64_peak}
        del pws, Cp
    # end to end through the public call: pinned host operands in, host result out
    if e2e_steps > 0:
        hA = torch.from_numpy(A).pin_memory()
        hB = torch.from_numpy(B).pin_memory()
        e2e_s = e2e_pipelined(torch, e2e_steps, [hA, hB],
                              lambda d: [mw.mw_gemm(d[0], d[1], plan, check=False)])
        mw.check_status()
        rec["e2e"] = {"value": aggregate(e2e_s, flops, 1, dist, dev)[0], "unit": "GFLOP/s",
                      "h2d_bytes_per_step": int(hA.numel() * 8 + hB.numel() * 8),
                      "d2h_bytes_per_step": int(m * M * N * 8),
                      "how": E2E_HOW + "; the plan made once before the loop"}
        del hA, hB
    if rank == 0 and cpu_s > 0:
        rec["cpu_baseline"] = cpu_sample(A, B, cpu_s, WORD_NAMES[m])
    del flush


def e2e_count(args):
    return args.e2e_steps if args.e2e_steps >= 0 else max(3, args.steps // 4)


def run_single(args, name, mw, torch, dist, rank, world, dev):
    """One of the single-product workloads on its own (profiling and sweeps)."""
    m, n, _, desc = WORKLOADS[name]
    if args.size:
        n = args.size
        desc = desc.replace("M=N=K=4096", f"M=N=K={n}").replace("M=N=K=1024", f"M=N=K={n}")
    A, B = single_inputs(name, args.size)
    pipes = measure_pipes(torch, dev)
    cpu_s = 0.0 if args.no_cpu else args.cpu_seconds
    rec = measure_single(args, mw, torch, dist, rank, dev, A, B, name, mode=args.mode,
                         graph=(not args.no_graph and n <= 1024), plain_steps=args.plain_steps,
                         e2e_steps=e2e_count(args), cpu_s=cpu_s, pipes=pipes)
    line = {"metric": METRIC, "value": rec["value"], "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(m, "exact integer residues" if args.mode == "crt" else
                              "exact integer slices") + "; bf16 operands on tcgen05",
            "data": "synthetic",
            "config": {"workload": desc, "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "fp64_peak_tflops_measured": pipes[0],
                       "int8_peak_tops_measured": pipes[1],
                       **{k: v for k, v in rec.items()
                          if k not in ("value", "unit", "roofline", "clocks", "e2e",
                                       "cpu_baseline", "gpu_launches", "workload")}},
            "roofline": rec["roofline"], "clocks": rec["clocks"], "e2e": rec.get("e2e"),
            "gpu_launches": rec["gpu_launches"]}
    if "cpu_baseline" in rec:
        line["cpu_baseline"] = rec["cpu_baseline"]
    return line


def autotune_record(mw, torch, tA, tB):
    """The autotuner's measured choice for these operands: every admissible
    (form, width, chunk) timed with CUDA events (mean of 3 after one untimed
    call, L2 not flushed), cached in a temporary file unless MW_AUTOTUNE_CACHE
    names one."""
    import tempfile
    from paper_2606_20863_gb300 import autotune
    path = os.environ.get("MW_AUTOTUNE_CACHE") or os.path.join(tempfile.mkdtemp(), "tune.json")
    tuner = autotune.Autotuner(path)
    choice, times = tuner.tune(tA, tB)
    torch.cuda.empty_cache()
    return {"choice": choice.as_dict(), "ms": {k: round(v, 3) for k, v in times.items()},
            "cache": "MW_AUTOTUNE_CACHE" if os.environ.get("MW_AUTOTUNE_CACHE") else "temporary"}


def run_headline(args, mw, torch, dist, rank, world, dev):
    """The benchmark line: quad double (value) and double double at 4096^3, each
    in both Ozaki forms (digit slices and residues) on the same operands and the
    same error bound, the faster one next to the plain FP64 form; quad double
    1024^3 as a secondary record."""
    import synthetic
    pipes = measure_pipes(torch, dev)
    cpu_s = 0.0 if args.no_cpu else args.cpu_seconds
    recs, best, tuned = {}, {}, {}
    for name, m in (("qd4096", 4), ("dd4096", 2)):
        A, B = synthetic.ozaki_4096(m)
        forms = {f: measure_single(args, mw, torch, dist, rank, dev, A, B, name, mode=f,
                                   pipes=pipes) for f in args.forms}
        win = max(forms, key=lambda f: forms[f]["value"])
        tA, tB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
        extras(args, mw, torch, dist, rank, dev, A, B, tA, tB, mw.plan_for(tA, tB, win),
               forms[win], args.plain_steps, e2e_count(args), cpu_s, pipes)
        if not args.no_autotune:
            tuned[name] = autotune_record(mw, torch, tA, tB)
        if "plain" in forms[win]:
            for f in forms:
                forms[f]["speedup_vs_plain"] = forms[f]["value"] / forms[win]["plain"]["value"]
        del tA, tB, A, B
        torch.cuda.empty_cache()
        best[name] = forms[win]
        for f, r in forms.items():
            recs[f"{name}_{f}"] = r
    if not args.no_secondary:
        A, B = synthetic.qd_1024()
        for f in args.forms:
            recs[f"qd1024_{f}"] = measure_single(args, mw, torch, dist, rank, dev, A, B, "qd1024",
                                                 mode=f, graph=not args.no_graph, pipes=pipes)
    qd = best["qd4096"]
    line = {"metric": METRIC, "value": qd["value"], "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": qd["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(4, "exact integer residues" if qd["mode"] == "crt" else
                              "exact integer slices") + "; bf16 operands on tcgen05",
            "data": "synthetic",
            "config": {"workload": HEADLINE, "m": [4, 2], "M": 4096, "N": 4096, "K": 4096,
                       "value_is": f"quad double 4096^3, Ozaki form '{qd['mode']}' (the faster "
                                   "of slices and residues), whole step (split, products, "
                                   "fusion), device-timed",
                       "dd4096_value": best["dd4096"]["value"],
                       "dd4096_form": best["dd4096"]["mode"],
                       "l2": "flushed (256 MiB write) before every timed step; operands "
                             "(1.6 GB quad double) also exceed L2",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "fp64_peak_tflops_measured": pipes[0],
                       "int8_peak_tops_measured": pipes[1],
                       "error_bound": "|C - C_exact| <= 2K 2^(-52m) (|A||B|) componentwise, "
                                      "every form (checked by the GPU tests)",
                       "autotune": tuned,
                       "records": recs},
            "roofline": qd["roofline"], "clocks": qd["clocks"], "e2e": qd.get("e2e"),
            "gpu_launches": qd["gpu_launches"]}
    if "cpu_baseline" in qd:
        line["cpu_baseline"] = qd["cpu_baseline"]
    return line


def run_batch(args, mw, torch, dist, rank, world, dev):
    """20,000 octo-double products, n ~ U{8..128}, seed 3, one batched call
    replayed from a CUDA graph per step."""
    import synthetic
    sizes = synthetic.batch_sizes(args.count, 8, 128, seed=3)
    FA, FB, offs = synthetic.batch_flat(sizes, m=8, seed=3)
    dA, dB = torch.from_numpy(FA).to(dev), torch.from_numpy(FB).to(dev)
    total = int(np.sum(sizes.astype(np.int64) ** 2))
    dC = torch.empty((8, total), dtype=torch.float64, device=dev)
    order = np.argsort(-sizes, kind="stable")          # largest problems first
    n_o = sizes[order].astype(np.int64)
    shapes = np.stack([n_o, n_o, n_o], axis=1)
    offsets = np.stack([offs[order]] * 3, axis=1)
    batch = mw.Batch.packed(dA, dB, dC, shapes, offsets)
    plan = batch.plan_
    flops = float(np.sum(2.0 * sizes.astype(np.float64) ** 3))
    pairs = count_pairs(plan)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    batch.run()
    torch.cuda.synchronize()
    mw.check_status()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.run()
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    step_ms, _, clk = timed(g.replay, args.steps, flush, mw, dist, dev, phase=False)
    value, t_step = aggregate(sum(step_ms) / 1e3, flops, args.steps, dist, dev)
    # product-kernel time: the same call launched directly (phase events are not
    # recorded inside a graph), as many runs as timed steps
    _, kern_ms, _ = timed(batch.run, max(3, args.steps), flush, mw, None, dev)
    phases = timed.phases
    roof = roofline_of(pairs, flops, kern_ms, "od_batch" if args.count == 20000 else None)
    roof["algorithmic"] = (f"{pairs} slice pairs x sum of 2 n^3 = {pairs * flops:.3e} flop per "
                           "launch; kernel time from direct calls of the batch")
    # end to end through the public API: pinned host operands in, every C_i out;
    # the batch is described and run per step with the plan made before the loop
    e2e_steps = args.e2e_steps if args.e2e_steps >= 0 else max(3, args.steps // 4)
    e2e = None
    if e2e_steps > 0:
        del batch, g, dC
        hA = torch.from_numpy(FA).pin_memory()
        hB = torch.from_numpy(FB).pin_memory()

        def batch_call(d):
            eC = torch.empty((8, total), dtype=torch.float64, device=dev)
            mw.Batch.packed(d[0], d[1], eC, shapes, offsets, plan).run()
            return [eC]
        e2e_s = e2e_pipelined(torch, e2e_steps, [hA, hB], batch_call)
        e2e = {"value": aggregate(e2e_s, flops, 1, dist, dev)[0], "unit": "GFLOP/s",
               "h2d_bytes_per_step": int((hA.numel() + hB.numel()) * 8),
               "d2h_bytes_per_step": int(8 * total * 8), "how": E2E_HOW}
        mw.check_status()
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(8),
            "data": "synthetic",
            "config": {"workload": f"{args.count:,} octo-double products, n ~ U{{8..128}} square, "
                                   "entries U[-1,1) with lower words x2^-53 U[-1,1), seed 3, one "
                                   "batched call replayed from a CUDA graph",
                       "m": 8, "count": args.count, "plan": plan.as_dict(), "slice_pairs": pairs,
                       "useful_flop_per_step": flops,
                       "phases_ms_direct_calls": phases,
                       "l2": "flushed (256 MiB write) before every timed step"},
            # prologue, lookup tables, item table, two splits, product, fusion
            "roofline": roof, "clocks": clk, "e2e": e2e, "gpu_launches": 7 * args.steps}
    if rank == 0 and not args.no_cpu:
        from oracle import textbook
        tc = textbook.TextbookC()
        from synthetic import SplitMix64
        pick = SplitMix64(5).next(400) % np.uint64(len(sizes))
        sample = [int(i) for i in pick]                  # 400 problems drawn with seed 5
        t0 = time.perf_counter()
        fl = 0.0
        for i in sample:
            n, o = int(sizes[i]), int(offs[i])
            a = np.ascontiguousarray(FA[:, o:o + n * n].reshape(8, n, n))
            b = np.ascontiguousarray(FB[:, o:o + n * n].reshape(8, n, n))
            tc.gemm(a, b)
            fl += 2.0 * n ** 3
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": fl / dt / 1e9, "unit": "GFLOP/s",
                                "cores": tc.max_threads(), "kind": "oracle",
                                "sample": f"400 of the {len(sizes):,} problems (SplitMix64 seed 5), {dt:.2f} s"}
    return line


def run_adjoint(args, mw, torch, dist, rank, world, dev):
    """Double-double A 2048 x 1024, B 1024 x 2048, W 2048 x 2048 (seed 4): one
    step is the forward product C = A B and the adjoint dA = W B^T, dB = A^T W
    through mw_gemm and mw_gemm_backward, all three in the Ozaki form."""
    import synthetic
    A, B, W = synthetic.adjoint_case()
    m, M, K = A.shape
    N = B.shape[2]
    Wm = np.zeros((m, M, N))
    Wm[0] = W
    tA, tB, tG = (torch.from_numpy(x).to(dev) for x in (A, B, Wm))
    pf = mw.plan_for(tA, tB, "ozaki")
    pa = mw.plan_for(tG, tB, "ozaki", False, True)
    pb = mw.plan_for(tA, tG, "ozaki", True, False)
    ws = torch.empty(mw.workspace_size(pf, M, N, K), dtype=torch.uint8, device=dev)
    C = torch.empty((m, M, N), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flops = 3 * 2.0 * M * N * K

    def step():
        mw.mw_gemm(tA, tB, pf, C=C, ws=ws, check=False)
        mw.mw_gemm_backward(tA, tB, tG, pa, pb, check=False)

    for _ in range(args.warmup):
        step()
    mw.check_status()
    torch.cuda.synchronize()
    step_ms, _, clk = timed(step, args.steps, flush, mw, dist, dev, phase=False)
    value, t_step = aggregate(sum(step_ms) / 1e3, flops, args.steps, dist, dev)

    # product-kernel time of each of the three products (phase events, own loop)
    calls = [(lambda c=None: mw.mw_gemm(tA, tB, pf, C=C, ws=ws, check=False), pf),
             (lambda: mw.mw_gemm(tG, tB, pa, transB=True, check=False), pa),
             (lambda: mw.mw_gemm(tA, tG, pb, transA=True, check=False), pb)]
    work, kern = 0.0, 0.0
    for f, pl in calls:
        _, kms, _ = timed(f, max(3, args.steps), flush, mw, None, dev)
        work += count_pairs(pl) * 2.0 * M * N * K
        kern += statistics.mean(kms)
    roof = roofline_of(1, work, [kern])
    roof["algorithmic"] = (f"forward, dA and dB: {count_pairs(pf)}, {count_pairs(pa)} and "
                           f"{count_pairs(pb)} slice pairs x {2.0 * M * N * K:.4g} flop; "
                           "achieved over the sum of the three product-kernel times")

    e2e_steps = args.e2e_steps if args.e2e_steps >= 0 else max(3, args.steps // 4)
    e2e = None
    if e2e_steps > 0:
        hA, hB, hW = (torch.from_numpy(x).pin_memory() for x in (A, B, Wm))

        def train_step(d):
            a = d[0].detach().requires_grad_(True)     # fresh leaves every step
            b = d[1].detach().requires_grad_(True)
            Cg = mw.MWGemm.apply(a, b)
            loss = (Cg * d[2]).sum(dim=(1, 2))       # per-plane sums: the loss's m words
            loss.sum().backward()
            return [loss.detach(), a.grad, b.grad]
        e2e_s = e2e_pipelined(torch, e2e_steps, [hA, hB, hW], train_step)
        e2e = {"value": aggregate(e2e_s, flops, 1, dist, dev)[0], "unit": "GFLOP/s",
               "h2d_bytes_per_step": int((hA.numel() + hB.numel() + hW.numel()) * 8),
               "d2h_bytes_per_step": int((m + hA.numel() + hB.numel()) * 8), "how": E2E_HOW}

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(2),
            "data": "synthetic",
            "config": {"workload": "double-double forward C=A*B and adjoint dA=W*B^T, dB=A^T*W, "
                                   "A 2048x1024, B 1024x2048, W 2048x2048, entries U[-1,1) with "
                                   "lower words x2^-53 U[-1,1), seed 4",
                       "m": m, "M": M, "N": N, "K": K,
                       "plans": {"forward": pf.as_dict(), "dA": pa.as_dict(), "dB": pb.as_dict()},
                       "flop_per_step": flops,
                       "l2": "flushed (256 MiB write) before every timed step"},
            "roofline": roof, "clocks": clk, "e2e": e2e,
            "gpu_launches": 3 * KERNELS_PER_STEP * args.steps}
    if rank == 0 and not args.no_cpu:
        from oracle import textbook
        tc = textbook.TextbookC()
        BT = np.ascontiguousarray(B.transpose(0, 2, 1))
        AT = np.ascontiguousarray(A.transpose(0, 2, 1))
        fl, t0 = 0.0, time.perf_counter()
        for X, Y in ((A, B), (Wm, BT), (AT, Wm)):
            tc.gemm(X, Y, threads=tc.max_threads())
            fl += 2.0 * X.shape[1] * X.shape[2] * Y.shape[2]
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": fl / dt / 1e9, "unit": "GFLOP/s",
                                "cores": tc.max_threads(), "kind": "oracle",
                                "sample": f"the whole step (C, dA and dB), {dt:.2f} s"}
    return line


# Table 2 of the paper: 1,024 inner products of length 6,144 on the Section 2 bit
# pattern, one thread of a Xeon 5318Y (milliseconds: ordinary, vectorized).
PAPER_TABLE2_MS = {2: (158.0, 69.0), 4: (1977.0, 318.0), 8: (6428.0, 1520.0),
                   16: (40780.0, 9491.0)}
# integer multiply-adds d_a d_b -> int64 per clock and SM assumed for the
# inner-product kernel's roofline (half the 128 int32 lanes of an SM)
IMAD_WIDE_PER_CLK_SM = 64


def run_table2(args, mw, torch, dist, rank, world, dev):
    """Table 2's workload on the GPU: 1,024 m-double inner products of length
    6,144, both vectors on the Section 2 bit pattern (seed 5), mw_dot_batched."""
    import synthetic
    m = args.m
    A, B = synthetic.table2_operands(m)
    _, count, K = A.shape
    tA, tB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    plan = mw.plan_dot(tA, tB)
    C = torch.empty((m, count), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flops = 2.0 * K * count

    def step():
        mw.mw_dot_batched(tA, tB, plan, C=C, check=False)

    for _ in range(args.warmup):
        step()
    mw.check_status()
    torch.cuda.synchronize()
    step_ms, _, clk = timed(step, args.steps, flush, mw, dist, dev, phase=False)
    value, t_step = aggregate(sum(step_ms) / 1e3, flops, args.steps, dist, dev)
    pairs = sum(1 for p in range(plan.S_A) for q in range(plan.S_B) if p + q < plan.D)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = nsm * IMAD_WIDE_PER_CLK_SM * (clk.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    kern_s = statistics.mean(step_ms) / 1e3
    achieved = pairs * K * count / kern_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T multiply-adds/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "dot_kernel (24-bit digits, int64 diagonal sums on the integer units)",
            "peak_source": f"{nsm} SMs x {IMAD_WIDE_PER_CLK_SM} int32 x int32 -> int64 "
                           "multiply-adds per clock x max SM clock (assumed rate)",
            "algorithmic": f"{pairs} digit pairs per entry x {K} x {count} per launch"}
    # the same kernel against HBM: every word of both vectors read once, the words
    # of every result written once
    _, _, hbm_gbs, hbm_src = load_peaks()
    bytes_alg = 2 * m * 8 * K * count + m * 8 * count
    roof["hbm"] = {"achieved": bytes_alg / kern_s / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                   "frac": bytes_alg / kern_s / 1e9 / hbm_gbs,
                   "peak_source": f"{hbm_src} copy bandwidth (MEASURED_PEAKS.json)",
                   "algorithmic": f"{bytes_alg} bytes per launch (every word of both vectors "
                                  "read once, the results written once)"}

    e2e_steps = args.e2e_steps if args.e2e_steps >= 0 else max(3, args.steps // 4)
    e2e = None
    if e2e_steps > 0:
        hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
        # the plan made before the loop, as a caller with fixed-range vectors would
        e2e_s = e2e_pipelined(torch, e2e_steps, [hA, hB],
                              lambda d: [mw.mw_dot_batched(d[0], d[1], plan, check=False)])
        e2e = {"value": aggregate(e2e_s, flops, 1, dist, dev)[0], "unit": "GFLOP/s",
               "h2d_bytes_per_step": int((hA.numel() + hB.numel()) * 8),
               "d2h_bytes_per_step": int(m * count * 8), "how": E2E_HOW}
        mw.check_status()
    ordinary, vectorized = PAPER_TABLE2_MS[m]
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(m, "24-bit integer digits, int64 sums"),
            "data": "synthetic",
            "config": {"workload": f"Table 2: {count} m-double inner products of length {K}, "
                                   "vectors on the Section 2 bit pattern, seed 5",
                       "m": m, "count": count, "K": K, "plan": plan.as_dict(),
                       "form": "MW_DOT: 24-bit digits, int64 diagonal sums, exact fusion",
                       "paper_table2_ms": {"ordinary": ordinary, "vectorized": vectorized,
                                           "hardware": "Xeon 5318Y, one thread"},
                       "speedup_vs_paper_vectorized": vectorized / (t_step * 1e3 / args.steps),
                       "l2": "flushed (256 MiB write) before every timed step"},
            "roofline": roof, "clocks": clk, "e2e": e2e, "gpu_launches": 1 * args.steps}
    if rank == 0 and not args.no_cpu:
        from oracle import textbook
        tc = textbook.TextbookC()
        t0 = time.perf_counter()
        for i in range(count):
            tc.gemm(np.ascontiguousarray(A[:, i:i + 1, :]),
                    np.ascontiguousarray(B[:, i:i + 1, :].transpose(0, 2, 1)), threads=1)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": flops / dt / 1e9, "unit": "GFLOP/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"all {count} inner products, one thread as in Table 2, "
                                          f"{dt:.2f} s"}
    return line


def run_series(args, mw, torch, dist, rank, world, dev):
    """Products of truncated power series: count pairs of octo-double series of
    degree 127 (n = 128 coefficients, entries U[-1,1) with lower words
    x2^-53 U[-1,1), seed 3), every coefficient c_i = sum_{k<=i} a_k b_(i-k) in one
    mw_convolve_batched call.  m-double flops: 2 sum_i (i+1) = n (n+1) a pair."""
    import synthetic
    m, n, count = 8, 128, args.count if args.count != 20000 else 2000
    rng = synthetic.SplitMix64(3)
    A = synthetic.uniform_mdouble(rng, m, count, n)
    B = synthetic.uniform_mdouble(rng, m, count, n)
    tA, tB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    plan = mw.plan_convolve(tA, tB)
    C = torch.empty((m, count, n), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flops = float(count) * n * (n + 1)

    def step():
        mw.mw_convolve_batched(tA, tB, plan, C=C, check=False)

    for _ in range(args.warmup):
        step()
    mw.check_status()
    torch.cuda.synchronize()
    step_ms, _, clk = timed(step, args.steps, flush, mw, dist, dev, phase=False)
    value, t_step = aggregate(sum(step_ms) / 1e3, flops, args.steps, dist, dev)
    e2e = None
    e2e_steps = e2e_count(args)
    if e2e_steps > 0:
        hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
        e2e_s = e2e_pipelined(torch, e2e_steps, [hA, hB],
                              lambda d: [mw.mw_convolve_batched(d[0], d[1], plan, check=False)])
        e2e = {"value": aggregate(e2e_s, flops, 1, dist, dev)[0], "unit": "GFLOP/s",
               "h2d_bytes_per_step": int((hA.numel() + hB.numel()) * 8),
               "d2h_bytes_per_step": int(m * count * n * 8), "how": E2E_HOW}
        mw.check_status()
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(m, "24-bit integer digits, int64 sums"), "data": "synthetic",
            "config": {"workload": f"{count} products of octo-double power series of degree "
                                   f"{n - 1}, entries U[-1,1) with lower words x2^-53 U[-1,1), "
                                   "seed 3, one mw_convolve_batched call",
                       "m": m, "count": count, "n": n, "plan": plan.as_dict(),
                       "flop_per_step": flops,
                       "l2": "flushed (256 MiB write) before every timed step"},
            "roofline": None, "clocks": clk, "e2e": e2e, "gpu_launches": args.steps}
    if rank == 0 and not args.no_cpu:
        from oracle import textbook
        tc = textbook.TextbookC()
        sample = min(count, 40)
        t0 = time.perf_counter()
        for s in range(sample):
            for i in range(n):
                a = np.ascontiguousarray(A[:, s:s + 1, :i + 1])
                b = np.ascontiguousarray(B[:, s, i::-1][:, :, None])
                tc.gemm(a, b, threads=1)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sample * n * (n + 1) / dt / 1e9, "unit": "GFLOP/s",
                                "cores": 1, "kind": "oracle",
                                "sample": f"{sample} of the {count} series products, one thread, "
                                          f"{dt:.2f} s"}
    return line


# FP64 instructions of one m-double operation on the GPU path (two_sum 6,
# fast_two_sum 3, two_prod 2 = a multiply and a fused multiply-add, a plain add or
# multiply 1, a division counted as 1), generic operands (every term nonzero), by
# stepping through the algorithms of mw_elementwise
ELEMENTWISE_FP64_OPS = {2: {"add": 20, "mul": 9, "div": 79},
                        4: {"add": 132, "mul": 515, "div": 2797},
                        8: {"add": 552, "mul": 3655, "div": 35225}}


def run_elementwise(args, mw, torch, dist, rank, world, dev):
    """Table 1's m-double add, mul or div entry by entry: 2^24 entries (division
    2^22, octo-double division 2^20; --count overrides), magnitudes 2^U[-20,20) random sign, lower words
    x2^-53 U[-1,1), seed 6, one mw_elementwise call.  Metric: m-double operations
    per second; roofline on the FP64 pipe (the instructions of one operation
    times the entries against half the measured DGEMM rate: one fused
    multiply-add is two flops), with the HBM view (three m-doubles an entry)."""
    import synthetic
    m, op = args.m, args.op
    if m not in ELEMENTWISE_FP64_OPS:
        raise SystemExit("elementwise: m = 2, 4 or 8")
    # default sizes: every launch well above L2 (129 MB), a step well under a second
    default_n = {"add": 1 << 24, "mul": 1 << 24, "div": 1 << 22 if m < 8 else 1 << 20}[op]
    n = args.count if args.count != 20000 else default_n
    rng = synthetic.SplitMix64(6)
    A = synthetic.loguniform_mdouble(rng, m, 1, n, -20, 20).reshape(m, n)
    B = synthetic.loguniform_mdouble(rng, m, 1, n, -20, 20).reshape(m, n)
    tA, tB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    C = torch.empty_like(tA)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        mw.mw_elementwise(op, tA, tB, C)

    fp64_peak, _ = measure_pipes(torch, dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    step_ms, _, clk = timed(step, args.steps, flush, mw, dist, dev, phase=False)
    value, t_step = aggregate(sum(step_ms) / 1e3, n, args.steps, dist, dev)   # G entries/s
    kern_s = statistics.mean(step_ms) / 1e3
    ops = ELEMENTWISE_FP64_OPS[m][op]
    achieved = ops * n / kern_s / 1e12
    peak = fp64_peak / 2
    _, _, hbm_gbs, hbm_src = load_peaks()
    bytes_alg = 3 * 8 * m * n
    roof = {"bound": "fp64", "achieved": achieved, "peak": peak,
            "unit": "T FP64 instructions/s", "frac": achieved / peak, "traffic": None,
            "kernel": f"elementwise_kernel<{m}, {op}> (textbook m-double arithmetic, FP64 pipe)",
            "peak_source": f"measured DGEMM rate {fp64_peak:.3f} TFLOP/s / 2 (cuBLAS, this run)",
            "algorithmic": f"{ops} FP64 instructions per entry x {n} entries per launch",
            "hbm": {"achieved": bytes_alg / kern_s / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                    "frac": bytes_alg / kern_s / 1e9 / hbm_gbs,
                    "peak_source": f"{hbm_src} copy bandwidth (MEASURED_PEAKS.json)",
                    "algorithmic": f"{bytes_alg} bytes per launch (A, B read, C written once)"}}
    e2e = None
    e2e_steps = e2e_count(args)
    if e2e_steps > 0:
        hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
        e2e_s = e2e_pipelined(torch, e2e_steps, [hA, hB],
                              lambda d: [mw.mw_elementwise(op, d[0], d[1])])
        e2e = {"value": aggregate(e2e_s, n, 1, dist, dev)[0],
               "unit": "G m-double operations/s",
               "h2d_bytes_per_step": int((hA.numel() + hB.numel()) * 8),
               "d2h_bytes_per_step": int(m * n * 8), "how": E2E_HOW}
    line = {"metric": f"m-double {op} operations per second (Table 1's {op}, entry by entry)",
            "value": value, "unit": "G m-double operations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"f64x{m} ({WORD_NAMES[m]}; FP64 operations)", "data": "synthetic",
            "config": {"workload": f"{n} {WORD_NAMES[m]} entries, {op}, magnitudes 2^U[-20,20) "
                                   "random sign, lower words x2^-53 U[-1,1), seed 6",
                       "m": m, "op": op, "n": n,
                       "l2": "inputs larger than L2, and flushed (256 MiB write) before every "
                             "timed step"},
            "roofline": roof, "clocks": clk, "e2e": e2e, "gpu_launches": args.steps}
    if rank == 0 and not args.no_cpu:
        from oracle import textbook
        tc = textbook.TextbookC()
        sample = min(n, 1 << 20 if op != "div" else 1 << 18)
        t0 = time.perf_counter()
        tc.elementwise(op, A[:, :sample], B[:, :sample])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sample / dt / 1e9, "unit": "G m-double operations/s",
                                "cores": tc.max_threads(), "kind": "oracle",
                                "sample": f"the first {sample} entries, {dt:.2f} s"}
    return line


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_2606_20863_gb300 as mw

    dist, rank, world = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.workload == "headline":
        line = run_headline(args, mw, torch, dist, rank, world, dev)
    elif args.workload == "od_batch":
        line = run_batch(args, mw, torch, dist, rank, world, dev)
    elif args.workload == "adjoint":
        line = run_adjoint(args, mw, torch, dist, rank, world, dev)
    elif args.workload == "table2":
        line = run_table2(args, mw, torch, dist, rank, world, dev)
    elif args.workload == "series":
        line = run_series(args, mw, torch, dist, rank, world, dev)
    elif args.workload == "elementwise":
        line = run_elementwise(args, mw, torch, dist, rank, world, dev)
    else:
        line = run_single(args, args.workload, mw, torch, dist, rank, world, dev)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
