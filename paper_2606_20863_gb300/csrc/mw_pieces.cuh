// Cutting one m-double entry into balanced pieces (device side, shared by the
// single and batched split kernels).
//   fixed_point: T = sum_j trunc(x_j 2^F) in NL 64-bit limbs, two's complement;
//   cut_pair:    the balanced base-2^w digits of two entries, least significant
//                first with a carry, stored as bfloat16 or double; raises
//                MW_ERANGE when T leaves [-2^(wS-1), 2^(wS-1)).
#pragma once
#include <cuda_bf16.h>

#include "mw_device.cuh"

namespace mw {
namespace {

// Fixed-point value of one entry in NL limbs (two's complement, little endian).
template <int MW, int NL>
__device__ __forceinline__ void fixed_point(const double (&w)[MW], int F, uint64_t (&T)[NL]) {
#pragma unroll
  for (int i = 0; i < NL; ++i) T[i] = 0;
#pragma unroll
  for (int j = 0; j < MW; ++j) {
    int e2;
    bool neg;
    uint64_t M = mantissa_of(w[j], e2, neg);
    if (M == 0) continue;
    const int sh = e2 + F;
    uint64_t lo = 0, hi = 0;
    int li = 0;
    if (sh < 0) {
      lo = (-sh) >= 64 ? 0 : (M >> (-sh));
      li = 0;
    } else {
      li = sh >> 6;
      const int off = sh & 63;
      lo = M << off;
      hi = off ? (M >> (64 - off)) : 0;
    }
    // T += (neg ? -1 : 1) * (hi:lo << 64*li), as T + (~V) + 1 when negative
    uint64_t carry = neg ? 1 : 0;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      uint64_t a = (i == li) ? lo : ((i == li + 1) ? hi : 0);
      if (neg) a = ~a;
      const uint64_t s1 = T[i] + a;
      const uint64_t c1 = s1 < a;
      const uint64_t s2 = s1 + carry;
      const uint64_t c2 = s2 < carry;
      T[i] = s2;
      carry = c1 | c2;
    }
  }
}

// Arithmetic right shift of the limbs by w (0 < w < 64).
template <int NL>
__device__ __forceinline__ void shr(uint64_t (&T)[NL], int w) {
#pragma unroll
  for (int i = 0; i < NL - 1; ++i) T[i] = (T[i] >> w) | (T[i + 1] << (64 - w));
  T[NL - 1] = (uint64_t)((int64_t)T[NL - 1] >> w);
}

template <typename Out>
__device__ __forceinline__ Out to_out(int d);
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(int d) {
  return __float2bfloat16_rn((float)d);  // |d| <= 2^(w-1) <= 256: exact
}
template <>
__device__ __forceinline__ double to_out<double>(int d) { return (double)d; }

template <typename Out>
__device__ __forceinline__ void store2(Out *p, int d0, int d1);
template <>
__device__ __forceinline__ void store2<__nv_bfloat16>(__nv_bfloat16 *p, int d0, int d1) {
  __nv_bfloat162 v;
  v.x = to_out<__nv_bfloat16>(d0);
  v.y = to_out<__nv_bfloat16>(d1);
  *reinterpret_cast<__nv_bfloat162 *>(p) = v;
}
template <>
__device__ __forceinline__ void store2<double>(double *p, int d0, int d1) {
  *reinterpret_cast<double2 *>(p) = make_double2((double)d0, (double)d1);
}

// Cut two entries (k, k+1 of one row) into S pieces and store them.
// w0, w1: the words of the two entries (zeros stand for entries past the row end).
template <int MW, int NL, typename Out>
__device__ __forceinline__ void cut_pair(const double (&w0)[MW], const double (&w1)[MW], int F,
                                         int w, int S, Out *dst, int64_t plane,
                                         unsigned int *status) {
  uint64_t T0[NL], T1[NL];
  fixed_point<MW, NL>(w0, F, T0);
  fixed_point<MW, NL>(w1, F, T1);
  const uint64_t mask = (1ull << w) - 1;
  const int half = 1 << (w - 1);
  int c0 = 0, c1 = 0;
  for (int p = S - 1; p >= 1; --p) {
    int r0 = (int)(T0[0] & mask) + c0, r1 = (int)(T1[0] & mask) + c1;
    c0 = r0 >= half;
    c1 = r1 >= half;
    r0 -= c0 << w;
    r1 -= c1 << w;
    store2<Out>(dst + p * plane, r0, r1);
    shr<NL>(T0, w);
    shr<NL>(T1, w);
  }
  // what is left is T >> w(S-1); T in [-2^(wS-1), 2^(wS-1)) <=> it lies in
  // [-2^(w-1), 2^(w-1)) with all higher limbs the sign extension of limb 0
  bool ok = true;
  const int64_t t0 = (int64_t)T0[0], t1 = (int64_t)T1[0];
#pragma unroll
  for (int i = 1; i < NL; ++i) {
    ok &= T0[i] == (uint64_t)(t0 >> 63);
    ok &= T1[i] == (uint64_t)(t1 >> 63);
  }
  ok &= t0 >= -half && t0 < half && t1 >= -half && t1 < half;
  if (!ok) raise_status(status, MW_ERANGE);
  store2<Out>(dst, (int)t0 + c0, (int)t1 + c1);
}

// The same for w = 8: the digits are the bytes of T (byte k = limb k/8, byte
// k%8, least significant first), so no multi-limb shifts are needed.
template <int MW, int NL, typename Out>
__device__ __forceinline__ void cut_pair_w8(const double (&w0)[MW], const double (&w1)[MW], int F,
                                            int S, Out *dst, int64_t plane, unsigned int *status) {
  uint64_t T0[NL], T1[NL];
  fixed_point<MW, NL>(w0, F, T0);
  fixed_point<MW, NL>(w1, F, T1);
  int c0 = 0, c1 = 0;
  bool ok = true;
  int top0 = 0, top1 = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * i + j;
      const int b0 = (int)((T0[i] >> (8 * j)) & 0xFF), b1 = (int)((T1[i] >> (8 * j)) & 0xFF);
      if (k < S - 1) {
        int r0 = b0 + c0, r1 = b1 + c1;
        c0 = r0 >= 128;
        c1 = r1 >= 128;
        r0 -= c0 << 8;
        r1 -= c1 << 8;
        store2<Out>(dst + (int64_t)(S - 1 - k) * plane, r0, r1);
      } else if (k == S - 1) {
        top0 = (int)(int8_t)b0;  // T >> 8(S-1) must be a signed byte
        top1 = (int)(int8_t)b1;
      } else {
        // bytes above the top digit: sign extension of the top byte
        ok &= b0 == (top0 < 0 ? 0xFF : 0) && b1 == (top1 < 0 ? 0xFF : 0);
      }
    }
  }
  if (!ok) raise_status(status, MW_ERANGE);
  store2<Out>(dst, top0 + c0, top1 + c1);
}

}  // namespace
}  // namespace mw
