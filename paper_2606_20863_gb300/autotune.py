"""Autotuner for the slicing of an m-double product.

The error analysis (``mw_plan_gemm``) fixes, for a given form and piece width,
how many pieces and diagonals a product needs; it does not say which form and
width run fastest on a given shape.  The tuner settles that by measurement:

* candidates: the residue form (m = 2 and 4) and the slice form with pieces of
  w = 6, 7 and 8 bits, each with the drain chunks its width allows (a sum of
  ``chunk`` products of w-bit balanced digits must stay below 2^24);
* every candidate is checked against the bound before it runs (``admissible``:
  the truncation of either operand and the dropped diagonals within their
  shares of 2K 2^(-52m), exact fp32 drains, a residue product P > 8 K
  2^(L_A + L_B - 2)); inadmissible plans are never timed;
* each admissible candidate is timed on the caller's operands (CUDA events on
  the current stream, after one untimed call), the fastest wins;
* the winner's form, width and chunk are cached per shape class (m, the powers
  of two bracketing M, N and K, the exponent spreads) in a JSON file, the path
  given by ``MW_AUTOTUNE_CACHE`` (default ``~/.cache/mw_autotune.json``); a later
  product of the class re-plans with the cached choice and the exact shape.

No counterpart in the paper: tile and slice choices are the library's.  The
bound the candidates must meet is the componentwise 2K 2^(-52m) (|A||B|) of
every form.
"""
from __future__ import annotations

import json
import math
import os
import threading
from dataclasses import dataclass

import torch

from . import (MWError, _dims, mw_crt_moduli_product_bits, mw_gemm, mw_measure_spread,
               mw_plan, mw_plan_gemm, workspace_size)

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("MW_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mw_autotune.json"))


def _bucket(x: int) -> int:
    """The power of two at or above x (shape classes)."""
    return 1 << max(0, math.ceil(math.log2(max(1, x))))


def shape_key(m: int, M: int, N: int, K: int, range_A: int, range_B: int) -> str:
    return f"m{m}/M{_bucket(M)}/N{_bucket(N)}/K{_bucket(K)}/rA{range_A}/rB{range_B}"


@dataclass(frozen=True)
class Choice:
    """What the tuner picks: the form ("crt" or "ozaki"), the piece width (slices)
    and the drain chunk (slices; 0 = the planner's)."""
    form: str
    w: int = 0
    chunk: int = 0

    def as_dict(self):
        return {"form": self.form, "w": self.w, "chunk": self.chunk}


def plan_of(choice: Choice, m: int, M: int, N: int, K: int, range_A: int,
            range_B: int) -> mw_plan:
    """The plan of a choice for an exact shape and spreads (the planner's counts)."""
    if choice.form == "crt":
        return mw_plan_gemm(m, "crt", M, N, K, range_A, range_B)
    p = mw_plan_gemm(m, "ozaki", M, N, K, range_A, range_B, choice.w)
    if choice.chunk:
        p.chunk = choice.chunk
    return p


def admissible(p: mw_plan, K: int) -> bool:
    """The plan meets the componentwise bound and keeps every sum exact (the
    shares of the error budget 2K 2^(-52m) the planner gives each source)."""
    m, lgK = p.m, math.log2(K)
    if p.mode == 3:                                           # residue form
        return (p.S_A >= 52 * m + p.range_A + math.log2(m) + 5 - lgK - 1e-9
                and p.S_B >= 52 * m + p.range_B + math.log2(m) + 5 - lgK - 1e-9
                and mw_crt_moduli_product_bits(p.D) > p.S_A + p.S_B + 1 + lgK)
    if p.mode != 1:
        return False
    w = p.w
    if not 2 <= w <= 8:
        return False
    if w * p.S_A < 52 * m + p.range_A + math.log2(m) + 5 - lgK - 1e-9:
        return False
    if w * p.S_B < 52 * m + p.range_B + math.log2(m) + 5 - lgK - 1e-9:
        return False
    if p.D < p.S_A + p.S_B - 1 and w * p.D < (52 * m + p.range_A + p.range_B
                                             + math.log2(min(p.S_A, p.S_B)) + 6 - lgK - 1e-9):
        return False
    return p.chunk >= 64 and p.chunk % 64 == 0 and p.chunk * 2 ** (2 * w - 2) <= 2 ** 24


def candidates(m: int, M: int, N: int, K: int, range_A: int, range_B: int) -> list[Choice]:
    out = []
    if m in (2, 4):
        out.append(Choice("crt"))
    for w in (8, 7, 6):
        top = (1 << 24) >> (2 * w - 2)                        # largest exact chunk
        for chunk in sorted({top, max(64, top // 4)}, reverse=True):
            out.append(Choice("ozaki", w, chunk))
    return [c for c in out
            if _try_plan(c, m, M, N, K, range_A, range_B) is not None]


def _try_plan(c, m, M, N, K, ra, rb):
    try:
        p = plan_of(c, m, M, N, K, ra, rb)
    except MWError:
        return None
    return p if admissible(p, K) else None


class Autotuner:
    """Measured choice of form, width and chunk per shape class, cached in JSON."""

    def __init__(self, path: str | None = None, reps: int = 3):
        self.path = path or cache_path()
        self.reps = reps
        self.table = self._load()
        self.last = None            # timings of the last tuning run

    def _load(self) -> dict:
        try:
            with open(self.path) as f:
                data = json.load(f)
            return data if isinstance(data, dict) else {}
        except (OSError, ValueError):
            return {}

    def _save(self):
        with _lock:
            d = os.path.dirname(self.path)
            if d:
                os.makedirs(d, exist_ok=True)
            tmp = f"{self.path}.{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    def cached(self, key: str) -> Choice | None:
        v = self.table.get(key)
        if not v:
            return None
        return Choice(v["form"], int(v.get("w", 0)), int(v.get("chunk", 0)))

    def record(self, key: str, choice: Choice, timings: dict | None = None):
        self.table[key] = dict(choice.as_dict(), **({"ms": timings} if timings else {}))
        self._save()

    def choose(self, m: int, M: int, N: int, K: int, range_A: int, range_B: int,
               time_fn) -> tuple[Choice, dict]:
        """Time every admissible candidate with time_fn(plan) -> milliseconds and
        cache the fastest for the shape class (host logic)."""
        times = {}
        for c in candidates(m, M, N, K, range_A, range_B):
            p = plan_of(c, m, M, N, K, range_A, range_B)
            times[json.dumps(c.as_dict(), sort_keys=True)] = float(time_fn(p))
        if not times:
            raise MWError("no admissible plan for this product")
        best = min(times, key=times.get)
        choice = Choice(**json.loads(best))
        self.record(shape_key(m, M, N, K, range_A, range_B), choice, times)
        self.last = times
        return choice, times

    def tune(self, A: torch.Tensor, B: torch.Tensor, transA=False,
             transB=False) -> tuple[Choice, dict]:
        """Time every admissible candidate on these operands (GPU) and cache the fastest."""
        m, M, N, K = _dims(A, B, transA, transB)
        ra, rb = mw_measure_spread(A, B, transA, transB)
        return self.choose(m, M, N, K, ra, rb,
                           lambda p: self._time(A, B, p, transA, transB, M, N, K))

    def _time(self, A, B, p, transA, transB, M, N, K) -> float:
        ws = torch.empty(workspace_size(p, M, N, K), dtype=torch.uint8, device=A.device)
        C = torch.empty((A.shape[0], M, N), dtype=torch.float64, device=A.device)
        mw_gemm(A, B, p, transA=transA, transB=transB, C=C, ws=ws)        # untimed, checked
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(self.reps):
            mw_gemm(A, B, p, transA=transA, transB=transB, C=C, ws=ws, check=False)
        ev[1].record()
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) / self.reps

    def plan_for(self, A: torch.Tensor, B: torch.Tensor, transA=False, transB=False) -> mw_plan:
        """The plan for this product: the cached choice of its shape class, tuned
        on these operands when the class has none (synchronizes)."""
        m, M, N, K = _dims(A, B, transA, transB)
        ra, rb = mw_measure_spread(A, B, transA, transB)
        choice = self.cached(shape_key(m, M, N, K, ra, rb))
        if choice is None:
            choice, _ = self.tune(A, B, transA, transB)
        p = plan_of(choice, m, M, N, K, ra, rb)
        if not admissible(p, K):
            raise MWError("cached choice is not admissible for this shape")
        return p
