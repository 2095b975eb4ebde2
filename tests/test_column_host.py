"""The column arithmetic of the CUDA library (cut_column, round_column in
csrc/mw_column.cuh) and its fusion of diagonal sums (csrc/mw_fuse.cuh),
compiled for the host with g++ (tests/column_host.cpp) and compared with the
oracle on seeded inputs: the balanced digits of T = sum_j trunc(x_j 2^F)
(Section 2's pieces on the shared grid) and its range check, the exact
integer sum_t s_t 2^(w (D-1-t)) of the diagonal sums, and the greedy
round-to-nearest words of an exact integer (Section 4's final
renormalisation).  No GPU; the device build of the same header is
checked by the GPU parity tests."""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact, slicing
from synthetic import SplitMix64, loguniform_mdouble, paper_pattern_mdouble, uniform_mdouble

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2606_20863_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("column") / "column_host")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-o", exe,
                    os.path.join(ROOT, "tests", "column_host.cpp")], check=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout.split("\n")
        return out[:len(lines)]
    return run


def hexbits(x: float) -> str:
    return "%016x" % struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def entries(m: int, n: int, seed: int):
    """Seeded m-doubles of several shapes, plus edge cases: powers of two (the
    top digit on the range edge), lone small words, zeros, sign changes."""
    rng = SplitMix64(seed)
    out = [list(uniform_mdouble(rng, m, 1, n)[:, 0, i]) for i in range(n)]
    out += [list(loguniform_mdouble(rng, m, 1, n, -30, 30)[:, 0, i]) for i in range(n)]
    out += [list(paper_pattern_mdouble(rng, m, 1, n)[:, 0, i]) for i in range(n)]
    r = random.Random(seed)
    for _ in range(n):
        e = r.randint(-40, 40)
        w = [math.ldexp(1.0, e) * r.choice([-1, 1])] + [0.0] * (m - 1)
        for j in range(1, m):
            if r.random() < 0.7:
                w[j] = math.ldexp(r.choice([-1, 1]) * (1 + r.random()), e - 53 * j - r.randint(1, 4))
        out.append(w)
    out.append([0.0] * m)
    out.append([-0.5] + [math.ldexp(1.0, -54 - 53 * j) for j in range(m - 1)])
    return out


CUT_CASES = [(8, 2, 15), (8, 4, 28), (8, 8, 56), (8, 16, 112),
             (24, 2, 5), (24, 4, 9), (24, 8, 17), (24, 16, 35)]


@pytest.mark.parametrize("w,m,S", CUT_CASES)
def test_cut_digits_equal_the_oracle(driver, w, m, S):
    lines, want = [], []
    r = random.Random(100 * w + m)
    for x in entries(m, 60, seed=1000 + 10 * m + w):
        E = slicing.entry_exponent(x)
        E = 0 if E is None else E
        # on the planner's grid, and (one in four) shifted off it to reach the range edges
        F = w * S - 2 - E + (r.randint(-2, 2) if r.random() < 0.25 else 0)
        T = slicing.fixed_point(x, F)
        ok = -(1 << (w * S - 1)) <= T < (1 << (w * S - 1))
        lines.append(f"cut {w} {S} {F} {m} " + " ".join(hexbits(v) for v in x))
        want.append((ok, slicing.balanced_digits(T, w, S) if ok else None))
    got = driver(lines)
    n_range = 0
    for line, (ok, digits), g in zip(lines, want, got):
        fields = g.split()
        assert fields[0] == ("ok" if ok else "range"), (line, g)
        if ok:
            assert [int(v) for v in fields[1:]] == digits, line
        else:
            n_range += 1
    assert 0 < n_range < len(lines)          # both outcomes exercised


@pytest.mark.parametrize("m,nl32", [(2, 8), (4, 12), (8, 20), (16, 34)])
def test_round_words_equal_the_oracle(driver, m, nl32):
    """Greedy words of X 2^ex for X in nl32 two's complement limbs, with every
    word in the normal range (the products' case)."""
    r = random.Random(7 * m + nl32)
    lines, want = [], []
    bits = 32 * nl32
    for i in range(300):
        kind = i % 5
        top = r.randint(1, bits - 2)
        if kind == 0:      # random
            X = r.getrandbits(top)
        elif kind == 1:    # runs of ones and zeros (carries through the negation)
            X = 0
            pos = 0
            while pos < top:
                run = r.randint(1, 70)
                if r.random() < 0.5:
                    X |= ((1 << run) - 1) << pos
                pos += run
            X &= (1 << top) - 1
        elif kind == 2:    # ties: a 53-bit head, then exactly half an ulp
            head = r.getrandbits(53) | (1 << 52)
            sh = r.randint(2, max(2, top - 53))
            X = (head << sh) | (1 << (sh - 1))
        elif kind == 3:    # sparse
            X = sum(1 << r.randint(0, top) for _ in range(r.randint(1, 6)))
        else:              # small
            X = r.getrandbits(r.randint(1, 60))
        if r.random() < 0.5:
            X = -X
        ex = -300 if bits < 700 else -600
        limbs = [(X >> (32 * k)) & 0xFFFFFFFF for k in range(nl32)]
        lines.append(f"round {m} {ex} {nl32} " + " ".join("%08x" % u for u in limbs))
        want.append([hexbits(v) for v in exact.greedy_words(Fraction(X) * Fraction(2) ** ex, m)])
    got = driver(lines)
    for line, wv, g in zip(lines, want, got):
        assert g.split() == wv, line


def test_small_integers_to_bfloat16_bits(driver):
    """The pieces' bfloat16 patterns: the top 16 bits of the float of d, every
    d in [-256, 256] (the balanced digits of w <= 9 bits)."""
    ds = list(range(-256, 257))
    got = driver([f"bf16 {d}" for d in ds])
    for d, g in zip(ds, got):
        b = struct.unpack("<I", struct.pack("<f", float(np.float32(d))))[0]
        assert b & 0xFFFF == 0
        assert int(g, 16) == b >> 16, d


@pytest.mark.parametrize("nl32,D", [(10, 30), (18, 60), (20, 72)])
def test_fusion_of_diagonal_sums_equals_the_oracle(driver, nl32, D):
    """X = sum_t s_t 2^(8 (D-1-t)) for int32 sums s_t, by the four-at-a-time
    Horner of fuse_w8 and by fuse_diagonals (groups of 1, 2, 4), against
    slicing.fuse_integer, as nl32 two's complement 32-bit limbs."""
    r = random.Random(nl32 * 100 + D)
    lines, want = [], []
    for i in range(200):
        kind = i % 4
        if kind == 0:
            sv = [r.randint(-2 ** 31, 2 ** 31 - 1) for _ in range(D)]
        elif kind == 1:
            sv = [r.choice([-2 ** 31, 2 ** 31 - 1, -1, 0, 1]) for _ in range(D)]
        elif kind == 2:
            sv = [r.randint(-2 ** 20, 2 ** 20) for _ in range(D)]
        else:
            sv = [0] * D
            sv[r.randrange(D)] = r.randint(-2 ** 31, 2 ** 31 - 1)
        g = (1, 2, 4)[i % 3]
        X = slicing.fuse_integer(sv, 8, D) % (1 << (32 * nl32))
        lines.append(f"fuse {g} {nl32} {D} " + " ".join(str(v) for v in sv))
        want.append(["%08x" % ((X >> (32 * k)) & 0xFFFFFFFF) for k in range(nl32)])
    got = driver(lines)
    for line, wv, g in zip(lines, want, got):
        a, b = g.split("|")
        assert a.split() == wv, line
        assert b.split() == wv, line
