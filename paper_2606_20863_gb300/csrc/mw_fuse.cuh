// Exact fusion of 64-bit partial sums and rounding to m words (device side,
// shared by the single and batched combine kernels).
//   add_shifted: X += V 2^sh on an NL-limb two's complement integer;
//   round_words: the m nonoverlapping doubles of X 2^ex, each the value
//                rounded to nearest (ties to even) of what the previous words
//                left over (greedy), computed on the exact integer.
#pragma once
#include <cstdint>

namespace mw {
namespace {

template <int NL>
__device__ __forceinline__ bool is_zero(const uint64_t (&x)[NL]) {
  uint64_t o = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i) o |= x[i];
  return o == 0;
}

// Shift left so that bit 63 of the top limb is set; returns the shift.
template <int NL>
__device__ __forceinline__ int normalize(uint64_t (&x)[NL]) {
  int sh = 0;
  // whole limbs first
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    if (x[NL - 1] == 0) {
#pragma unroll
      for (int i = NL - 1; i > 0; --i) x[i] = x[i - 1];
      x[0] = 0;
      sh += 64;
    }
  }
  const int b = __clzll((long long)x[NL - 1]);
  if (b) {
#pragma unroll
    for (int i = NL - 1; i > 0; --i) x[i] = (x[i] << b) | (x[i - 1] >> (64 - b));
    x[0] <<= b;
  }
  return sh + b;
}

template <int NL>
__device__ __forceinline__ void add_shifted(uint64_t (&X)[NL], int64_t V, int sh) {
  const int li = sh >> 6, bo = sh & 63;
  const uint64_t lo = (uint64_t)V << bo;
  const uint64_t hi = bo ? (uint64_t)(V >> (64 - bo)) : (uint64_t)(V >> 63);
  const uint64_t ext = (uint64_t)(V >> 63);
  uint64_t carry = 0;
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const uint64_t a = k < li ? 0 : (k == li ? lo : (k == li + 1 ? hi : ext));
    const uint64_t s1 = X[k] + a;
    const uint64_t c1 = s1 < a;
    const uint64_t s2 = s1 + carry;
    const uint64_t c2 = s2 < carry;
    X[k] = s2;
    carry = c1 | c2;
  }
}

// X += sum_t s_t 2^(w (D-1-t)) for the int32 diagonal sums s_t = p[t * plane]:
// 32 independent loads at a time, then Horner in int64 over each group of
// `group` consecutive diagonals (exact for the planner's group size) and one
// multi-limb add per group.
template <int NL>
__device__ __forceinline__ void fuse_diagonals(uint64_t (&X)[NL], const int32_t *p, int64_t plane,
                                               int D, int group, int w) {
  int64_t V = 0;
  int in_group = 0;
  for (int t0 = 0; t0 < D; t0 += 32) {
    int32_t s[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) s[u] = (t0 + u < D) ? p[(int64_t)(t0 + u) * plane] : 0;
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      const int t = t0 + u;
      if (t < D) {
        V = (int64_t)((uint64_t)V << w) + s[u];
        if (++in_group == group || t == D - 1) {
          add_shifted<NL>(X, V, w * (D - 1 - t));
          V = 0;
          in_group = 0;
        }
      }
    }
  }
}

template <int MW, int NL>
__device__ __forceinline__ void round_words(uint64_t (&X)[NL], int ex, double (&words)[MW]) {
#pragma unroll
  for (int k = 0; k < MW; ++k) words[k] = 0.0;
  // magnitude and sign
  bool neg = (int64_t)X[NL - 1] < 0;
  if (neg) {
    uint64_t c = 1;
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const uint64_t s = ~X[k] + c;
      c = (s == 0 && c) ? 1 : 0;
      X[k] = s;
    }
  }
#pragma unroll
  for (int k = 0; k < MW; ++k) {
    if (is_zero<NL>(X)) break;
    ex -= normalize<NL>(X);
    const uint64_t top = X[NL - 1];
    uint64_t mant = top >> 11;
    const uint64_t rbit = (top >> 10) & 1;
    uint64_t sticky = top & 0x3FF;
#pragma unroll
    for (int q = 0; q < NL - 1; ++q) sticky |= X[q];
    const uint64_t up = rbit & ((sticky != 0) | (mant & 1));
    mant += up;
    const double mag = scalbn((double)mant, ex + 64 * (NL - 1) + 11);
    words[k] = neg ? -mag : mag;
    // remainder: low bits minus (up ? 2^pos : 0), pos = 64 (NL-1) + 11
    X[NL - 1] = top & 0x7FF;
    if (up) {
      // X <- 2^pos - low, and the sign flips
      X[NL - 1] = (~X[NL - 1]) & 0x7FF;
#pragma unroll
      for (int q = 0; q < NL - 1; ++q) X[q] = ~X[q];
      uint64_t c = 1;
#pragma unroll
      for (int q = 0; q < NL; ++q) {
        const uint64_t s = X[q] + c;
        c = (s == 0 && c) ? 1 : 0;
        X[q] = s;
      }
      neg = !neg;
    }
  }
}

}  // namespace
}  // namespace mw
