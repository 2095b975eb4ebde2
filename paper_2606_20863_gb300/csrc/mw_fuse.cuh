// Exact fusion of the partial sums (device side,
// shared by the single and batched combine kernels).
//   add_shifted:    X += V 2^sh on an NL-limb (64-bit) two's complement integer;
//   fuse_diagonals: X += sum_t s_t 2^(w (D-1-t)), any w, 64-bit limbs;
//   fuse_w8:        the same sum for w = 8 straight into 32-bit limbs
// (the rounding of X into m words is round_column in mw_column.cuh).  All of it
// compiles for the host too (checked against the oracle there).
#pragma once
#include <cstdint>

#include "mw_column.cuh"   // MW_HD: host and device (plain integer code)

namespace mw {
namespace {

template <int NL>
MW_HD void add_shifted(uint64_t (&X)[NL], int64_t V, int sh) {
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

// X += sum_t s_t 2^(w (D-1-t)) for the int32 diagonal sums s_t = p[t * plane]
// (any w): 8 independent loads at a time, then Horner in int64 over each group
// of `group` consecutive diagonals (exact for the planner's group size) and one
// multi-limb add per group.
template <int NL>
MW_HD void fuse_diagonals(uint64_t (&X)[NL], const int32_t *p, int64_t plane,
                                               int D, int group, int w) {
  int64_t V = 0;
  int in_group = 0;
  for (int t0 = 0; t0 < D; t0 += 8) {
    int32_t s[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) s[u] = (t0 + u < D) ? p[(int64_t)(t0 + u) * plane] : 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
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

// The same integer as 2 NL 32-bit limbs (two's complement).
template <int NL>
MW_HD void to_limbs32(const uint64_t (&X)[NL], uint32_t (&U)[2 * NL]) {
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    U[2 * k] = (uint32_t)X[k];
    U[2 * k + 1] = (uint32_t)(X[k] >> 32);
  }
}

// X = sum_t s_t 2^(8 (D-1-t)) for w = 8 and the int32 diagonal sums
// s_t = p[t * plane], as NL32 32-bit limbs (two's complement), built from the
// least significant end: limb j takes the four sums of weights 2^(32j),
// 2^(32j+8), 2^(32j+16), 2^(32j+24), joined by Horner in 64 bits (|.| < 2^56),
// plus the signed carry out of limb j-1.  The sums are loaded sixteen at a time
// (four limbs), so that more loads are in flight.
template <int NL32>
MW_HD void fuse_w8(uint32_t (&U)[NL32], const int32_t *p, int64_t plane,
                                        int D) {
  static_assert(NL32 % 2 == 0, "limbs in pairs");
  const int32_t *last = p + (int64_t)(D - 1) * plane;   // s_{D-1}, weight 2^0
  int64_t R = 0;
#pragma unroll
  for (int j = 0; j < NL32; j += 4) {
    int32_t s[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int u = 4 * j + k;                            // s_{D-1-u}, weight 2^(8u)
      s[k] = (u < D && j + k / 4 < NL32) ? last[-(int64_t)u * plane] : 0;
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      if (j + h >= NL32) break;
      int64_t V = s[4 * h + 3];
      V = V * 256 + s[4 * h + 2];
      V = V * 256 + s[4 * h + 1];
      V = V * 256 + s[4 * h];
      R += V;
      U[j + h] = (uint32_t)R;
      R >>= 32;
    }
  }
}

}  // namespace
}  // namespace mw
