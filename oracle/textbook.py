"""Textbook m-double arithmetic (oracle part O1; test infrastructure only).

Two renderings of the same textbook algorithms (described in ``textbook.c``):

* ``TextbookC``  -- ctypes front end of ``textbook.c``, compiled with gcc
  ``-O2 -ffp-contract=off -fopenmp``; the timed CPU baseline.
* ``Counting``   -- the same steps in Python on IEEE doubles, counting every
  floating-point operation; reproduces the operation counts of Table 1 for
  double-double addition and gives this file's counts for the rest.

Python floats are IEEE doubles with round-to-nearest and no fused
multiply-add, so both renderings must agree bit for bit.

Parity unpinned: ``op_counts`` for the m-double multiplication (m = 2: 24
operations where Table 1 prints 23) and for m = 4, 8, 16 (Table 1's counts
belong to algorithms the paper does not give); the counts of the double-double
addition are pinned to Table 1.  Division: the paper gives only its operation
count (Table 1), so ``div`` / ``tb_div`` are this project's long division; their
results are pinned by exact rational arithmetic (a relative error bound against
a / b) and exact cases, their counts are not pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmwtextbook.so")
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile textbook.c into oracle/_build/libmwtextbook.so (gcc, OpenMP).
    The textbook m-double arithmetic of Section 1 and Table 1, in C."""
    with _lock:
        src = os.path.join(_HERE, "textbook.c")
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(src)):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _SO)
        return _SO


class TextbookC:
    """Textbook m-double GEMM in C (Section 1's arithmetic, the operation counts of Table 1)."""
    def __init__(self):
        self.lib = ctypes.CDLL(build())
        i64, dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        self.lib.tb_gemm_rows.argtypes = [ctypes.c_int, i64, i64, i64, dp, dp, dp,
                                          ctypes.POINTER(i64), i64, ctypes.c_int]
        self.lib.tb_mul.argtypes = [ctypes.c_int, dp, dp, dp]
        self.lib.tb_add.argtypes = [ctypes.c_int, dp, dp, dp]
        self.lib.tb_div.argtypes = [ctypes.c_int, dp, dp, dp]
        self.lib.tb_elementwise.argtypes = [ctypes.c_int, ctypes.c_int, i64, dp, dp, dp,
                                            ctypes.c_int]
        self.lib.tb_max_threads.restype = ctypes.c_int

    @staticmethod
    def _p(a: np.ndarray):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def max_threads(self) -> int:
        """Threads the C oracle runs on (OpenMP)."""
        return self.lib.tb_max_threads()

    def gemm(self, A: np.ndarray, B: np.ndarray, rows: Sequence[int] | None = None,
             threads: int | None = None) -> np.ndarray:
        """C = A B (m, M, N); only ``rows`` are computed when given (others stay 0).
        Textbook m-double GEMM (Section 1's arithmetic, Table 1's 'ordinary' inner products)."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        m, M, K = A.shape
        _, K2, N = B.shape
        assert K == K2 and B.shape[0] == m and m in (2, 4, 8, 16)
        C = np.zeros((m, M, N))
        r = np.arange(M, dtype=np.int64) if rows is None else np.asarray(rows, dtype=np.int64)
        self.lib.tb_gemm_rows(m, M, N, K, self._p(A), self._p(B), self._p(C),
                              r.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(r),
                              threads or self.max_threads())
        return C

    def elementwise(self, name: str, A: np.ndarray, B: np.ndarray,
                    threads: int | None = None) -> np.ndarray:
        """C = A op B entry by entry, op in add, mul, div; A, B (m, ...) m-double
        arrays.  Table 1's m-double add, mul and div."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        assert A.shape == B.shape and A.shape[0] in (2, 4, 8, 16)
        m = A.shape[0]
        n = A.size // m
        C = np.zeros_like(A)
        self.lib.tb_elementwise({"add": 0, "mul": 1, "div": 2}[name], m, n, self._p(A),
                                self._p(B), self._p(C), threads or self.max_threads())
        return C

    def op(self, name: str, a: Sequence[float], b: Sequence[float]) -> list[float]:
        """One m-double add, multiply or divide in C (Section 1's arithmetic; Table 1)."""
        m = len(a)
        x = np.array(a, dtype=np.float64)
        y = np.array(b, dtype=np.float64)
        r = np.zeros(m)
        getattr(self.lib, "tb_" + name)(m, self._p(x), self._p(y), self._p(r))
        return list(r)


class Counting:
    """The textbook algorithms in Python, counting floating-point operations.
    Section 1 and Table 1."""

    def __init__(self):
        self.flops = 0

    def _f(self, n: int = 1):
        self.flops += n

    def two_sum(self, a, b):
        """Error-free sum of two doubles (Section 1's arithmetic; Table 1 counts its 6 operations)."""
        s = a + b
        bv = s - a
        av = s - bv
        e = (a - av) + (b - bv)
        self._f(6)
        return s, e

    def fast_two_sum(self, a, b):
        """Error-free sum when |a| >= |b| (Section 1's arithmetic; 3 operations)."""
        s = a + b
        e = b - (s - a)
        self._f(3)
        return s, e

    def split(self, a):
        """Dekker's split of a double into two halves (for two_prod without fused multiply-add)."""
        c = 134217729.0 * a
        hi = c - (c - a)
        lo = a - hi
        self._f(4)
        return hi, lo

    def two_prod(self, a, b):
        """Error-free product of two doubles (Dekker; Section 1's arithmetic)."""
        p = a * b
        self._f(1)
        ah, al = self.split(a)
        bh, bl = self.split(b)
        e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
        self._f(8)
        return p, e

    def dd_add(self, a, b):
        """Double double addition (Section 1; Table 1: 20 operations)."""
        s, e = self.two_sum(a[0], b[0])
        t, f = self.two_sum(a[1], b[1])
        e = e + t
        self._f(1)
        s, e = self.fast_two_sum(s, e)
        e = e + f
        self._f(1)
        s, e = self.fast_two_sum(s, e)
        return [s, e]

    def dd_mul(self, a, b):
        """Double double multiplication (Section 1; Table 1: 23 operations)."""
        p, e = self.two_prod(a[0], b[0])
        e = e + (a[0] * b[1] + a[1] * b[0])
        self._f(4)
        p, e = self.fast_two_sum(p, e)
        return [p, e]

    def renorm(self, x, m):
        """Renormalisation of m + 1 words into m nonoverlapping words (Section 1's arithmetic)."""
        x = list(x)
        r = []
        for _ in range(m):
            if not x:
                r.append(0.0)
                continue
            s = x[-1]
            errs = [0.0] * len(x)
            for i in range(len(x) - 2, -1, -1):
                s, e = self.two_sum(x[i], s)
                errs[i + 1] = e
            r.append(s)
            x = [e for e in errs[1:] if e != 0.0]
        return r

    def add(self, a, b):
        """m-double addition (Section 1's arithmetic)."""
        m = len(a)
        if m == 2:
            return self.dd_add(a, b)
        t = []
        for i in range(m):
            t += [a[i], b[i]]
        return self.renorm(t, m)

    def mul(self, a, b):
        """m-double multiplication (Section 1's arithmetic)."""
        m = len(a)
        if m == 2:
            return self.dd_mul(a, b)
        t, lo_prev = [], []
        for l in range(m):
            lo_cur = []
            for i in range(l + 1):
                p, e = self.two_prod(a[i], b[l - i])
                t.append(p)
                lo_cur.append(e)
            t += lo_prev
            lo_prev = lo_cur
        for i in range(1, m):
            t.append(a[i] * b[m - i])
            self._f(1)
        t += lo_prev
        return self.renorm(t, m)

    def div(self, a, b):
        """m-double division a / b by long division (Table 1's div; the paper gives
        only its operation count): m + 1 quotient words, each the leading word of
        the remainder over b's leading word, the remainder reduced by q_i b (an
        m-double product and addition, for m >= 4 renormalised once more) after
        each of the first m, then the quotient words renormalised into m."""
        m = len(a)
        rem, q = list(a), []
        for i in range(m + 1):
            qi = rem[0] / b[0]
            self._f(1)
            q.append(qi)
            if i == m:
                break
            t = self.mul([qi] + [0.0] * (m - 1), b)
            rem = self.add(rem, [-x for x in t])
            if m > 2:                # the sum cancels in its leading words: once more
                rem = self.renorm(rem, m)
        return self.renorm(q, m)

    def gemm(self, A: np.ndarray, B: np.ndarray) -> np.ndarray:
        """Textbook m-double GEMM (Section 1's arithmetic, Table 1's 'ordinary' inner products)."""
        m, M, K = A.shape
        N = B.shape[2]
        C = np.zeros((m, M, N))
        for i in range(M):
            for j in range(N):
                acc = [0.0] * m
                for k in range(K):
                    p = self.mul([float(A[w, i, k]) for w in range(m)],
                                 [float(B[w, k, j]) for w in range(m)])
                    acc = self.add(acc, p)
                C[:, i, j] = acc
        return C


def op_counts(m: int, trials: int = 1) -> tuple[int, int]:
    """(flops of one m-double add, flops of one m-double mul) on nonzero operands.
    The renormalisation of m >= 4 drops exact-zero terms, so its count is that
    of generic (all terms nonzero) operands.
    Table 1: operations per m-double add and multiply."""
    from synthetic import SplitMix64, uniform_mdouble
    X = uniform_mdouble(SplitMix64(7), m, 1, 2)
    a = [float(X[j, 0, 0]) for j in range(m)]
    b = [float(X[j, 0, 1]) for j in range(m)]
    c = Counting()
    c.add(a, b)
    n_add = c.flops
    c.flops = 0
    c.mul(a, b)
    return n_add, c.flops
