"""Python binding of libmw, the GB300 m-double matrix product library.

Argument marshalling only: every step of the product runs in the CUDA kernels
of ``libmw.so`` (C interface ``include/mw.h``); PyTorch supplies device memory
and the current stream.  An m-double matrix is a float64 tensor of shape
(m, rows, cols) whose last dimension is contiguous; plane j holds word j of
every entry (m = 2, 4, 8 or 16).

The functions keep the names of the C entry points: ``mw_plan_gemm``,
``mw_split``, ``mw_gemm``, ``mw_gemm_backward``; ``MWGemm`` is the
``torch.autograd.Function`` over ``mw_gemm`` / ``mw_gemm_backward``.
If the compiled library is missing this module raises on import: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmw.so")

MW_OK, MW_EINVAL, MW_ERANGE, MW_ENONFINITE, MW_ECUDA, MW_ETIMEOUT, MW_ENOSPC, MW_WRANGE = (
    0, 1, 2, 4, 8, 16, 32, 64)
MW_PLAIN, MW_OZAKI, MW_DOT, MW_CRT, MW_TEXTBOOK = 0, 1, 2, 3, 4
MW_DIGITS_BF16, MW_DIGITS_F64 = 0, 1
_MODES = {"plain": MW_PLAIN, "ozaki": MW_OZAKI, "dot": MW_DOT, "crt": MW_CRT,
          "textbook": MW_TEXTBOOK}
STATUS_NAMES = {MW_ERANGE: "ERANGE", MW_ENONFINITE: "ENONFINITE", MW_ETIMEOUT: "ETIMEOUT",
                MW_WRANGE: "WRANGE"}


class MWError(RuntimeError):
    pass


class MWRangeError(MWError):
    """An operand's exponent spread exceeded the spread its plan was made for
    (status bit MW_WRANGE): the result is computed, but the componentwise error
    bound is no longer guaranteed.  Replan (``plan_for``) for such operands."""


class mw_plan(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("m", "mode", "w", "S_A", "S_B", "D", "group", "chunk", "range_A", "range_B")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}

    def __repr__(self):
        return "mw_plan(" + ", ".join(f"{k}={v}" for k, v in self.as_dict().items()) + ")"


class mw_problem(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("plane_stride_a", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("plane_stride_b", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64), ("plane_stride_c", ctypes.c_int64)]


class mw_batch(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int)] + [(n, ctypes.c_int64) for n in
                ("sum_M", "sum_N", "sum_MN", "max_M", "max_N", "min_K", "max_K")]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(_LIB_PATH)
    i64, i32, vp, ip = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(mw_plan)
    sig = {
        "mw_plan_gemm": [i32, i32, i64, i64, i64, i32, i32, pp],
        "mw_split": [i32, i32, i64, i64, vp, i64, i64, i32, i32, i32, vp, i64, vp, vp, vp, i32, vp],
        "mw_gemm_workspace_size": [pp, i64, i64, i64, ctypes.POINTER(ctypes.c_size_t)],
        "mw_gemm_workspace_layout": [pp, i64, i64, i64, ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t)],
        "mw_gemm": [pp, i32, i32, i64, i64, i64, vp, i64, i64, vp, i64, i64, vp, i64, i64,
                    vp, ctypes.c_size_t, vp],
        "mw_gemm_noalloc": [pp, i32, i32, i64, i64, i64, vp, i64, i64, vp, i64, i64, vp, i64,
                            i64, vp],
        "mw_measure_spread": [i32, i32, i32, i64, i64, i64, vp, i64, i64, vp, i64, i64, vp,
                              ctypes.c_size_t, ip, ip, vp],
        "mw_gemm_backward": [pp, pp, i64, i64, i64, vp, i64, i64, vp, i64, i64, vp, i64, i64,
                             vp, i64, i64, vp, i64, i64, vp, ctypes.c_size_t, vp],
        "mw_get_status": [ip, i32],
        "mw_batch_describe": [i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(mw_batch)],
        "mw_gemm_batched_workspace_size": [pp, ctypes.POINTER(mw_batch),
                                           ctypes.POINTER(ctypes.c_size_t)],
        "mw_measure_spread_batched": [i32, ctypes.POINTER(mw_batch), vp, vp, ctypes.c_size_t,
                                      ip, ip, vp],
        "mw_measure_spread_batched_workspace_size": [i32, ctypes.POINTER(mw_batch),
                                                     ctypes.POINTER(ctypes.c_size_t)],
        "mw_gemm_batched": [pp, ctypes.POINTER(mw_batch), vp, vp, ctypes.c_size_t, vp],
        "mw_dot_batched": [pp, i64, i64, vp, i64, i64, vp, i64, i64, vp, i64, vp],
        "mw_selftest_timeout": [ctypes.c_uint, vp],
        "mw_crt_moduli": [ip, i32],
        "mw_convolve_batched": [pp, i64, i64, vp, i64, i64, vp, i64, i64, vp, i64, i64, vp],
        "mw_set_phase_events": [ctypes.POINTER(ctypes.c_void_p), i32],
        "mw_elementwise": [i32, i32, i64, vp, i64, vp, i64, vp, i64, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.mw_last_error.restype = ctypes.c_char_p
    lib.mw_version.restype = ctypes.c_char_p
    return lib


_lib = _load()
LIB_PATH = _LIB_PATH
EXPORTED = ("mw_plan_gemm", "mw_split", "mw_gemm_workspace_size", "mw_gemm_workspace_layout",
            "mw_gemm",
            "mw_measure_spread", "mw_gemm_backward", "mw_get_status", "mw_last_error",
            "mw_version", "mw_set_phase_events", "mw_gemm_noalloc", "mw_batch_describe",
            "mw_gemm_batched_workspace_size", "mw_measure_spread_batched",
            "mw_measure_spread_batched_workspace_size", "mw_gemm_batched",
            "mw_dot_batched", "mw_selftest_timeout", "mw_crt_moduli", "mw_convolve_batched",
            "mw_elementwise")


def _check(rc: int, what: str):
    if rc != MW_OK:
        raise MWError(f"{what} failed ({rc}): {_lib.mw_last_error().decode()}")


def version() -> str:
    return _lib.mw_version().decode()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _mat(X: torch.Tensor, name: str):
    """(pointer, ld, plane_stride) of an (m, rows, cols) float64 CUDA tensor whose
    rows are contiguous (strides of dimensions of size 1 do not matter)."""
    if X.dtype != torch.float64 or X.dim() != 3 or not X.is_cuda:
        raise MWError(f"{name} must be a CUDA float64 tensor of shape (m, rows, cols)")
    rows, cols = X.shape[1], X.shape[2]
    if cols > 1 and X.stride(2) != 1:
        raise MWError(f"{name}: last dimension must be contiguous")
    ld = X.stride(1) if rows > 1 else cols
    if ld < cols:
        raise MWError(f"{name}: rows overlap (stride {ld} < {cols} columns)")
    return ctypes.c_void_p(X.data_ptr()), ld, X.stride(0)


def set_phase_events(events=None):
    """Record torch.cuda.Event objects (4 of them) between the phases of every
    mw_gemm: before the pieces, before the product kernel, after it, at the end."""
    if events is None:
        _check(_lib.mw_set_phase_events(None, 0), "mw_set_phase_events")
        return
    for e in events:            # torch creates the CUDA event on its first record
        if not e.cuda_event:
            e.record()
    arr = (ctypes.c_void_p * 4)(*[ctypes.c_void_p(e.cuda_event) for e in events])
    _check(_lib.mw_set_phase_events(arr, 4), "mw_set_phase_events")


def get_status(clear: bool = True) -> int:
    """Status bits raised by kernels on the current device (synchronizes)."""
    bits = ctypes.c_int(0)
    _check(_lib.mw_get_status(ctypes.byref(bits), int(clear)), "mw_get_status")
    return bits.value


def check_status(allow: int = 0):
    """Raise if a kernel reported an error bit other than those in ``allow``
    (synchronizes).  MW_WRANGE alone raises MWRangeError: a reused plan met
    operands of a wider exponent spread than it was made for, so the error
    bound is not guaranteed; pass ``allow=MW_WRANGE`` to accept that."""
    bits = get_status(clear=True)
    bad = bits & ~allow
    if bad:
        names = [n for b, n in STATUS_NAMES.items() if bits & b]
        msg = f"kernel status {bits}: {', '.join(names)}"
        if bad == MW_WRANGE:
            raise MWRangeError(msg + " (an operand's exponent spread exceeds the plan's; the "
                               "error bound is not guaranteed: replan with plan_for)")
        raise MWError(msg)
    return bits


def crt_moduli(n: int | None = None) -> list[int]:
    """The residue form's moduli in the order plans use them (the first n)."""
    total = _lib.mw_crt_moduli(None, 0)
    n = total if n is None else min(n, total)
    buf = (ctypes.c_int * max(n, 1))()
    _lib.mw_crt_moduli(buf, n)
    return list(buf[:n])


def mw_crt_moduli_product_bits(n: int) -> float:
    """log2 of the product of the first n moduli of the residue form."""
    import math
    return sum(math.log2(p) for p in crt_moduli(n))


def mw_plan_gemm(m: int, mode: str | int, M: int, N: int, K: int, range_A: int,
                 range_B: int, w: int = 0) -> mw_plan:
    p = mw_plan()
    p.w = w
    mode = _MODES.get(mode, mode)
    _check(_lib.mw_plan_gemm(m, mode, M, N, K, range_A, range_B, ctypes.byref(p)),
           "mw_plan_gemm")
    return p


def workspace_size(plan: mw_plan, M: int, N: int, K: int) -> int:
    n = ctypes.c_size_t(0)
    _check(_lib.mw_gemm_workspace_size(ctypes.byref(plan), M, N, K, ctypes.byref(n)),
           "mw_gemm_workspace_size")
    return n.value


def workspace_layout(plan: mw_plan, M: int, N: int, K: int):
    """(offsets of exponents, pieces of A, pieces of B, partial sums; total bytes)."""
    off = (ctypes.c_size_t * 4)()
    n = ctypes.c_size_t(0)
    _check(_lib.mw_gemm_workspace_layout(ctypes.byref(plan), M, N, K, off, ctypes.byref(n)),
           "mw_gemm_workspace_layout")
    return list(off), n.value


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def _dims(A, B, transA, transB):
    m = A.shape[0]
    M, K = (A.shape[2], A.shape[1]) if transA else (A.shape[1], A.shape[2])
    Kb, N = (B.shape[2], B.shape[1]) if transB else (B.shape[1], B.shape[2])
    if K != Kb or B.shape[0] != m:
        raise MWError(f"shape mismatch: op(A) {M}x{K}, op(B) {Kb}x{N}, m {m}/{B.shape[0]}")
    return m, M, N, K


def mw_measure_spread(A: torch.Tensor, B: torch.Tensor, transA=False, transB=False):
    """Exponent spreads of the rows of op(A) and the columns of op(B) (synchronizes)."""
    m, M, N, K = _dims(A, B, transA, transB)
    ws = _workspace(4 * (2 * M + 2 * N + 2), A.device)
    ra, rb = ctypes.c_int(0), ctypes.c_int(0)
    pa, lda, psa = _mat(A, "A")
    pb, ldb, psb = _mat(B, "B")
    _check(_lib.mw_measure_spread(m, int(transA), int(transB), M, N, K, pa, lda, psa, pb, ldb,
                                  psb, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                  ctypes.byref(ra), ctypes.byref(rb), _stream()),
           "mw_measure_spread")
    return ra.value, rb.value


def mw_split(X: torch.Tensor, w: int, S: int, trans: bool = False, fmt: str = "bf16",
             range_: int = -1):
    """Cut the logical operand (rows x K; X stored rows x K, or K x rows when
    ``trans``) into S pieces of w bits.  Returns (digits, exps, spread):
    digits (S, rows, Kp) bfloat16 or float64 with Kp = K rounded up to 64."""
    m = X.shape[0]
    R, K = (X.shape[2], X.shape[1]) if trans else (X.shape[1], X.shape[2])
    Kp = (K + 63) // 64 * 64
    dtype = torch.bfloat16 if fmt == "bf16" else torch.float64
    digits = torch.empty((S, R, Kp), dtype=dtype, device=X.device)
    exps = torch.empty(R, dtype=torch.int32, device=X.device)
    spread = torch.empty(R, dtype=torch.int32, device=X.device)
    px, ld, ps = _mat(X, "X")
    _check(_lib.mw_split(m, int(trans), R, K, px, ld, ps, w, S,
                         MW_DIGITS_BF16 if fmt == "bf16" else MW_DIGITS_F64,
                         ctypes.c_void_p(digits.data_ptr()), Kp,
                         ctypes.c_void_p(exps.data_ptr()), ctypes.c_void_p(spread.data_ptr()),
                         None, range_, _stream()), "mw_split")
    return digits, exps, spread


def plan_for(A: torch.Tensor, B: torch.Tensor, mode="ozaki", transA=False, transB=False,
             **overrides) -> mw_plan:
    """Plan with the exponent spreads measured on the operands (synchronizes)."""
    m, M, N, K = _dims(A, B, transA, transB)
    ra, rb = mw_measure_spread(A, B, transA, transB)
    p = mw_plan_gemm(m, mode, M, N, K, ra, rb, overrides.pop("w", 0))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def mw_gemm(A: torch.Tensor, B: torch.Tensor, plan: mw_plan | None = None, mode="ozaki",
            transA=False, transB=False, C: torch.Tensor | None = None,
            ws: torch.Tensor | None = None, check: bool = True) -> torch.Tensor:
    """C = op(A) op(B) in m-double precision."""
    m, M, N, K = _dims(A, B, transA, transB)
    if plan is None:
        plan = plan_for(A, B, mode, transA, transB)
    if C is None:
        C = torch.empty((m, M, N), dtype=torch.float64, device=A.device)
    need = workspace_size(plan, M, N, K)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, A.device)
    pa, lda, psa = _mat(A, "A")
    pb, ldb, psb = _mat(B, "B")
    pc, ldc, psc = _mat(C, "C")
    _check(_lib.mw_gemm(ctypes.byref(plan), int(transA), int(transB), M, N, K, pa, lda, psa,
                        pb, ldb, psb, pc, ldc, psc, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                        _stream()), "mw_gemm")
    if check:
        check_status()
    return C


def mw_gemm_noalloc(A: torch.Tensor, B: torch.Tensor, plan: mw_plan, transA=False,
                    transB=False, C: torch.Tensor | None = None) -> torch.Tensor:
    """mw_gemm without a workspace argument, for callers that cannot allocate
    device memory: the library's fixed per-device scratch (32 MiB) is used;
    larger products raise.  C, if given, must be preallocated by the caller."""
    m, M, N, K = _dims(A, B, transA, transB)
    if C is None:
        C = torch.empty((m, M, N), dtype=torch.float64, device=A.device)
    pa, lda, psa = _mat(A, "A")
    pb, ldb, psb = _mat(B, "B")
    pc, ldc, psc = _mat(C, "C")
    _check(_lib.mw_gemm_noalloc(ctypes.byref(plan), int(transA), int(transB), M, N, K, pa, lda,
                                psa, pb, ldb, psb, pc, ldc, psc, _stream()), "mw_gemm_noalloc")
    return C


def mw_gemm_backward(A: torch.Tensor, B: torch.Tensor, G: torch.Tensor,
                     plan_dA: mw_plan | None = None, plan_dB: mw_plan | None = None,
                     mode="ozaki", need_dA=True, need_dB=True, check: bool = True):
    """dA = G B^T and dB = A^T G for C = A B (A M x K, B K x N, G M x N)."""
    m, M, K = A.shape
    N = B.shape[2]
    if plan_dA is None and need_dA:
        plan_dA = plan_for(G, B, mode, False, True)
    if plan_dB is None and need_dB:
        plan_dB = plan_for(A, G, mode, True, False)
    need = max(workspace_size(plan_dA, M, K, N) if need_dA else 0,
               workspace_size(plan_dB, K, N, M) if need_dB else 0)
    ws = _workspace(need, A.device)
    dA = torch.empty((m, M, K), dtype=torch.float64, device=A.device) if need_dA else None
    dB = torch.empty((m, K, N), dtype=torch.float64, device=A.device) if need_dB else None
    pa, lda, psa = _mat(A, "A")
    pb, ldb, psb = _mat(B, "B")
    pg, ldg, psg = _mat(G, "G")
    pda, ldda, psda = _mat(dA, "dA") if need_dA else (None, 0, 0)
    pdb, lddb, psdb = _mat(dB, "dB") if need_dB else (None, 0, 0)
    _check(_lib.mw_gemm_backward(ctypes.byref(plan_dA) if need_dA else None,
                                 ctypes.byref(plan_dB) if need_dB else None, M, N, K,
                                 pa, lda, psa, pb, ldb, psb, pg, ldg, psg,
                                 pda, ldda, psda, pdb, lddb, psdb,
                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream()),
           "mw_gemm_backward")
    if check:
        check_status()
    return dA, dB


class Batch:
    """A batch of independent products C_i = A_i B_i, every matrix an m-double
    CUDA tensor (m, rows, cols).  Holds the device array of descriptors, the
    plan and the workspace, so that ``run()`` can be captured in a CUDA graph
    and replayed while the tensors keep their addresses."""

    def __init__(self, As, Bs, Cs=None, plan: mw_plan | None = None):
        if len(As) != len(Bs) or not As:
            raise MWError("need equally many A and B, at least one")
        self.m = As[0].shape[0]
        dev = As[0].device
        self.As, self.Bs = As, Bs
        self.Cs = Cs if Cs is not None else [
            torch.empty((self.m, a.shape[1], b.shape[2]), dtype=torch.float64, device=dev)
            for a, b in zip(As, Bs)]
        count = len(As)
        host = (mw_problem * count)()
        shapes = np.empty((count, 3), dtype=np.int64)
        for i, (a, b, c) in enumerate(zip(As, Bs, self.Cs)):
            if a.shape[2] != b.shape[1] or a.shape[0] != self.m or b.shape[0] != self.m:
                raise MWError(f"problem {i}: shape mismatch")
            pa, lda, psa = _mat(a, "A")
            pb, ldb, psb = _mat(b, "B")
            pc, ldc, psc = _mat(c, "C")
            host[i] = mw_problem(a.shape[1], b.shape[2], a.shape[2], pa.value, lda, psa,
                                 pb.value, ldb, psb, pc.value, ldc, psc)
            shapes[i] = (a.shape[1], b.shape[2], a.shape[2])
        self._setup(bytes(host), shapes, dev, plan)

    @classmethod
    def packed(cls, A, B, C, shapes, offsets, plan: mw_plan | None = None):
        """A batch whose matrices lie back to back in three flat m-plane tensors
        A, B, C of shape (m, total) (contiguous rows, ld = columns): problem i
        is (M_i, N_i, K_i) = shapes[i], its A_i, B_i, C_i start at element
        offsets[i] = (oA, oB, oC) of every plane.  Descriptors are built without
        a per-problem Python loop."""
        self = cls.__new__(cls)
        self.m = A.shape[0]
        for X in (A, B, C):
            if X.dim() != 2 or X.dtype != torch.float64 or X.stride(1) != 1 or X.shape[0] != self.m:
                raise MWError("packed operands are (m, total) float64 tensors, unit column stride")
        shapes = np.ascontiguousarray(shapes, dtype=np.int64).reshape(-1, 3)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64).reshape(-1, 3)
        M, N, K = shapes[:, 0], shapes[:, 1], shapes[:, 2]
        oA, oB, oC = offsets[:, 0], offsets[:, 1], offsets[:, 2]
        if (shapes < 1).any() or (oA < 0).any() or (oB < 0).any() or (oC < 0).any() or \
                (oA + M * K > A.shape[1]).any() or (oB + K * N > B.shape[1]).any() or \
                (oC + M * N > C.shape[1]).any():
            raise MWError("packed batch: a problem lies outside its flat tensor")
        d = np.empty((len(shapes), 12), dtype=np.int64)
        d[:, 0], d[:, 1], d[:, 2] = M, N, K
        d[:, 3], d[:, 4], d[:, 5] = A.data_ptr() + 8 * oA, K, A.stride(0)
        d[:, 6], d[:, 7], d[:, 8] = B.data_ptr() + 8 * oB, N, B.stride(0)
        d[:, 9], d[:, 10], d[:, 11] = C.data_ptr() + 8 * oC, N, C.stride(0)
        self.As, self.Bs, self.Cs = A, B, C
        self._setup(d.tobytes(), shapes, A.device, plan)
        return self

    def _setup(self, desc: bytes, shapes: np.ndarray, dev, plan):
        count = len(shapes)
        sh = np.ascontiguousarray(shapes, dtype=np.int64).reshape(-1)
        self.batch = mw_batch()
        _check(_lib.mw_batch_describe(count, sh.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      ctypes.byref(self.batch)), "mw_batch_describe")
        raw = torch.frombuffer(bytearray(desc), dtype=torch.uint8)
        self.d_problems = raw.to(dev)
        if plan is None:
            plan = self.plan()
        self.plan_ = plan
        n = ctypes.c_size_t(0)
        _check(_lib.mw_gemm_batched_workspace_size(ctypes.byref(plan), ctypes.byref(self.batch),
                                                   ctypes.byref(n)),
               "mw_gemm_batched_workspace_size")
        self.ws = _workspace(n.value, dev)

    def measure_spread(self):
        """Largest exponent spreads over the batch (synchronizes)."""
        b = self.batch
        need = ctypes.c_size_t(0)
        _check(_lib.mw_measure_spread_batched_workspace_size(self.m, ctypes.byref(b),
                                                             ctypes.byref(need)),
               "mw_measure_spread_batched_workspace_size")
        ws = _workspace(need.value, self.d_problems.device)
        ra, rb = ctypes.c_int(0), ctypes.c_int(0)
        _check(_lib.mw_measure_spread_batched(self.m, ctypes.byref(b),
                                              ctypes.c_void_p(self.d_problems.data_ptr()),
                                              ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                              ctypes.byref(ra), ctypes.byref(rb), _stream()),
               "mw_measure_spread_batched")
        return ra.value, rb.value

    def plan(self) -> mw_plan:
        """Plan for every problem: slice counts from the smallest K (tightest bound),
        diagonal groups that fit the largest K."""
        ra, rb = self.measure_spread()
        b = self.batch
        p = mw_plan_gemm(self.m, "ozaki", b.max_M, b.max_N, b.min_K, ra, rb)
        p.group = min(p.group, mw_plan_gemm(self.m, "ozaki", b.max_M, b.max_N, b.max_K, ra,
                                            rb).group)
        return p

    def run(self):
        _check(_lib.mw_gemm_batched(ctypes.byref(self.plan_), ctypes.byref(self.batch),
                                    ctypes.c_void_p(self.d_problems.data_ptr()),
                                    ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                    _stream()), "mw_gemm_batched")
        return self.Cs


def mw_gemm_batched(As, Bs, Cs=None, plan: mw_plan | None = None, check: bool = True):
    """C_i = A_i B_i for every i in one batched call (Ozaki form)."""
    b = Batch(As, Bs, Cs, plan)
    out = b.run()
    if check:
        check_status()
    return out


class MWGemm(torch.autograd.Function):
    """C = A B for m-double tensors (m, rows, cols).  The gradient with respect
    to an m-double input is the m-double value of dL/dA in the same plane
    format (not a derivative per plane): dA = G B^T, dB = A^T G."""

    @staticmethod
    def forward(ctx, A, B, mode="ozaki"):
        ctx.save_for_backward(A, B)
        ctx.mode = mode
        return mw_gemm(A, B, mode=mode)

    @staticmethod
    def backward(ctx, G):
        A, B = ctx.saved_tensors
        G = G.contiguous()
        dA, dB = mw_gemm_backward(A, B, G, mode=ctx.mode, need_dA=ctx.needs_input_grad[0],
                                  need_dB=ctx.needs_input_grad[1])
        return dA, dB, None


def plan_dot(A: torch.Tensor, B: torch.Tensor) -> mw_plan:
    """MW_DOT plan for the inner products of the rows of A and B, both
    (m, count, K), with the exponent spreads measured on them (synchronizes)."""
    m, count, K = A.shape
    ra, rb = mw_measure_spread(A, B, False, True)
    return mw_plan_gemm(m, "dot", 1, 1, K, ra, rb)


def mw_dot_batched(A: torch.Tensor, B: torch.Tensor, plan: mw_plan | None = None,
                   C: torch.Tensor | None = None, check: bool = True) -> torch.Tensor:
    """c_i = sum_k A[:, i, k] B[:, i, k] in m-double precision for every row i;
    A and B are (m, count, K), the result (m, count)."""
    if A.dim() != 3 or B.shape != A.shape:
        raise MWError("A and B must be (m, count, K) tensors of one shape")
    m, count, K = A.shape
    if plan is None:
        plan = plan_dot(A, B)
    if C is None:
        C = torch.empty((m, count), dtype=torch.float64, device=A.device)
    pa, lda, psa = _mat(A, "A")
    pb, ldb, psb = _mat(B, "B")
    if C.dtype != torch.float64 or not C.is_cuda or C.shape != (m, count) or C.stride(1) != 1:
        raise MWError("C must be a CUDA float64 (m, count) tensor with unit column stride")
    _check(_lib.mw_dot_batched(ctypes.byref(plan), count, K, pa, lda, psa, pb, ldb, psb,
                               ctypes.c_void_p(C.data_ptr()), C.stride(0), _stream()),
           "mw_dot_batched")
    if check:
        check_status()
    return C


MW_OP_ADD, MW_OP_MUL, MW_OP_DIV = 0, 1, 2
_OPS = {"add": MW_OP_ADD, "mul": MW_OP_MUL, "div": MW_OP_DIV}


def mw_elementwise(op: str, A: torch.Tensor, B: torch.Tensor,
                   C: torch.Tensor | None = None) -> torch.Tensor:
    """C = A op B entry by entry (op "add", "mul" or "div"; Table 1's m-double
    operations); A, B and C are contiguous CUDA float64 tensors of one shape
    (m, ...), plane j = A[j]."""
    if op not in _OPS:
        raise MWError(f"op must be add, mul or div, not {op!r}")
    if A.shape != B.shape or A.dim() < 2:
        raise MWError("A and B must be (m, ...) tensors of one shape")
    if C is None:
        C = torch.empty_like(A)
    for name, t in (("A", A), ("B", B), ("C", C)):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.shape != A.shape:
            raise MWError(f"{name} must be a contiguous CUDA float64 tensor of A's shape")
    m = A.shape[0]
    n = A[0].numel()
    _check(_lib.mw_elementwise(_OPS[op], m, n, ctypes.c_void_p(A.data_ptr()), n,
                               ctypes.c_void_p(B.data_ptr()), n, ctypes.c_void_p(C.data_ptr()), n,
                               _stream()), "mw_elementwise")
    return C


def plan_convolve(A: torch.Tensor, B: torch.Tensor) -> mw_plan:
    """MW_DOT plan for the products of the series in the rows of A and B, both
    (m, count, n): one inner product of length 1 (the shortest coefficient needs
    the most bits) with the exponent spreads of whole rows (a coefficient's
    vectors span no more), measured on the GPU (synchronizes)."""
    m = A.shape[0]
    ra, rb = mw_measure_spread(A, B, False, True)
    return mw_plan_gemm(m, "dot", 1, 1, 1, ra, rb)


def mw_convolve_batched(A: torch.Tensor, B: torch.Tensor, plan: mw_plan | None = None,
                        C: torch.Tensor | None = None, check: bool = True) -> torch.Tensor:
    """Products of truncated power series: C[:, s, i] = sum_{k<=i} A[:, s, k] B[:, s, i-k]
    in m-double precision; A and B are (m, count, n), the result (m, count, n)."""
    if A.dim() != 3 or B.shape != A.shape:
        raise MWError("A and B must be (m, count, n) tensors of one shape")
    m, count, n = A.shape
    if plan is None:
        plan = plan_convolve(A, B)
    if C is None:
        C = torch.empty((m, count, n), dtype=torch.float64, device=A.device)
    pa, lda, psa = _mat(A, "A")
    pb, ldb, psb = _mat(B, "B")
    pc, ldc, psc = _mat(C, "C")
    _check(_lib.mw_convolve_batched(ctypes.byref(plan), count, n, pa, lda, psa, pb, ldb, psb,
                                    pc, ldc, psc, _stream()), "mw_convolve_batched")
    if check:
        check_status()
    return C


def selftest_timeout(limit_us: int = 50000) -> int:
    """Let one bounded wait run out on the GPU (a barrier nothing completes) and
    return the status bits it left (MW_ETIMEOUT expected); synchronizes."""
    get_status(clear=True)
    _check(_lib.mw_selftest_timeout(limit_us, _stream()), "mw_selftest_timeout")
    return get_status(clear=True)
