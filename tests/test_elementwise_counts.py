"""The FP64 instruction counts behind the elementwise workload's roofline
(`bench.ELEMENTWISE_FP64_OPS`), recounted by stepping through the oracle's
textbook add, mul and div with the GPU's costs: two_prod is a multiply and a
fused multiply-add (2), two_sum 6, fast_two_sum 3, a plain add, multiply or
division 1, and the renormalisation sweeps keep zero terms (fixed-size arrays,
as in the kernels).  CPU only."""
from fractions import Fraction

import pytest

import bench
from oracle import textbook
from synthetic import SplitMix64, uniform_mdouble


class GpuCounting(textbook.Counting):
    def two_prod(self, a, b):
        p = a * b
        self._f(2)
        return p, float(Fraction(a) * Fraction(b) - Fraction(p))

    def renorm(self, x, m):
        x, r = list(x), []
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
            x = errs[1:]
        return r


@pytest.mark.parametrize("m", [2, 4, 8])
def test_elementwise_instruction_counts(m):
    X = uniform_mdouble(SplitMix64(7), m, 1, 2)
    a = [float(X[j, 0, 0]) for j in range(m)]
    b = [float(X[j, 0, 1]) for j in range(m)]
    for op in ("add", "mul", "div"):
        c = GpuCounting()
        getattr(c, op)(a, b)
        assert c.flops == bench.ELEMENTWISE_FP64_OPS[m][op], (m, op)
