// Cutting one m-double entry into balanced pieces (device side, shared by the
// single and batched split kernels).
//   fixed_point: T = sum_j trunc(x_j 2^F) in NL 64-bit limbs, two's complement;
//   cut_pair:    the balanced base-2^w digits of two entries, least significant
//                first with a carry, stored as bfloat16 or double; raises
//                MW_ERANGE when T leaves [-2^(wS-1), 2^(wS-1));
//   cut_one, cut_one_w8: the same for one entry (w = 8: digits straight from
//                the bytes of T plus a bias, no carry chain).
#pragma once
#include <cuda_bf16.h>

#include "mw_column.cuh"
#include "mw_device.cuh"

namespace mw {
namespace {

// T += A and T -= A on NL 64-bit limbs, one carry chain of add.cc/addc
// (sub.cc/subc) instructions.
template <int NL>
__device__ __forceinline__ void add_limbs(uint64_t (&T)[NL], const uint64_t (&A)[NL]) {
  uint64_t c = 0;   // the same arithmetic for other compilers
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const uint64_t s1 = T[i] + A[i], c1 = s1 < A[i];
    const uint64_t s2 = s1 + c;
    c = c1 | (s2 < c);
    T[i] = s2;
  }
}
template <int NL>
__device__ __forceinline__ void sub_limbs(uint64_t (&T)[NL], const uint64_t (&A)[NL]) {
  uint64_t b = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const uint64_t d1 = T[i] - A[i], b1 = T[i] < A[i];
    const uint64_t d2 = d1 - b;
    b = b1 | (d1 < b);
    T[i] = d2;
  }
}
#if defined(__CUDA_ARCH__)
template <>
__device__ __forceinline__ void add_limbs<2>(uint64_t (&T)[2], const uint64_t (&A)[2]) {
  asm("{\n"
      "add.cc.u64 %0, %0, %2;\n"
      "addc.u64 %1, %1, %3;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1])
      : "l"(A[0]), "l"(A[1]));
}
template <>
__device__ __forceinline__ void sub_limbs<2>(uint64_t (&T)[2], const uint64_t (&A)[2]) {
  asm("{\n"
      "sub.cc.u64 %0, %0, %2;\n"
      "subc.u64 %1, %1, %3;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1])
      : "l"(A[0]), "l"(A[1]));
}
template <>
__device__ __forceinline__ void add_limbs<4>(uint64_t (&T)[4], const uint64_t (&A)[4]) {
  asm("{\n"
      "add.cc.u64 %0, %0, %4;\n"
      "addc.cc.u64 %1, %1, %5;\n"
      "addc.cc.u64 %2, %2, %6;\n"
      "addc.u64 %3, %3, %7;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1]), "+l"(T[2]), "+l"(T[3])
      : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]));
}
template <>
__device__ __forceinline__ void sub_limbs<4>(uint64_t (&T)[4], const uint64_t (&A)[4]) {
  asm("{\n"
      "sub.cc.u64 %0, %0, %4;\n"
      "subc.cc.u64 %1, %1, %5;\n"
      "subc.cc.u64 %2, %2, %6;\n"
      "subc.u64 %3, %3, %7;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1]), "+l"(T[2]), "+l"(T[3])
      : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]));
}
template <>
__device__ __forceinline__ void add_limbs<6>(uint64_t (&T)[6], const uint64_t (&A)[6]) {
  asm("{\n"
      "add.cc.u64 %0, %0, %6;\n"
      "addc.cc.u64 %1, %1, %7;\n"
      "addc.cc.u64 %2, %2, %8;\n"
      "addc.cc.u64 %3, %3, %9;\n"
      "addc.cc.u64 %4, %4, %10;\n"
      "addc.u64 %5, %5, %11;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1]), "+l"(T[2]), "+l"(T[3]), "+l"(T[4]), "+l"(T[5])
      : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]));
}
template <>
__device__ __forceinline__ void sub_limbs<6>(uint64_t (&T)[6], const uint64_t (&A)[6]) {
  asm("{\n"
      "sub.cc.u64 %0, %0, %6;\n"
      "subc.cc.u64 %1, %1, %7;\n"
      "subc.cc.u64 %2, %2, %8;\n"
      "subc.cc.u64 %3, %3, %9;\n"
      "subc.cc.u64 %4, %4, %10;\n"
      "subc.u64 %5, %5, %11;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1]), "+l"(T[2]), "+l"(T[3]), "+l"(T[4]), "+l"(T[5])
      : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]));
}
template <>
__device__ __forceinline__ void add_limbs<8>(uint64_t (&T)[8], const uint64_t (&A)[8]) {
  asm("{\n"
      "add.cc.u64 %0, %0, %8;\n"
      "addc.cc.u64 %1, %1, %9;\n"
      "addc.cc.u64 %2, %2, %10;\n"
      "addc.cc.u64 %3, %3, %11;\n"
      "addc.cc.u64 %4, %4, %12;\n"
      "addc.cc.u64 %5, %5, %13;\n"
      "addc.cc.u64 %6, %6, %14;\n"
      "addc.u64 %7, %7, %15;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1]), "+l"(T[2]), "+l"(T[3]), "+l"(T[4]), "+l"(T[5]), "+l"(T[6]), "+l"(T[7])
      : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(A[7]));
}
template <>
__device__ __forceinline__ void sub_limbs<8>(uint64_t (&T)[8], const uint64_t (&A)[8]) {
  asm("{\n"
      "sub.cc.u64 %0, %0, %8;\n"
      "subc.cc.u64 %1, %1, %9;\n"
      "subc.cc.u64 %2, %2, %10;\n"
      "subc.cc.u64 %3, %3, %11;\n"
      "subc.cc.u64 %4, %4, %12;\n"
      "subc.cc.u64 %5, %5, %13;\n"
      "subc.cc.u64 %6, %6, %14;\n"
      "subc.u64 %7, %7, %15;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1]), "+l"(T[2]), "+l"(T[3]), "+l"(T[4]), "+l"(T[5]), "+l"(T[6]), "+l"(T[7])
      : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(A[7]));
}
template <>
__device__ __forceinline__ void add_limbs<10>(uint64_t (&T)[10], const uint64_t (&A)[10]) {
  asm("{\n"
      "add.cc.u64 %0, %0, %10;\n"
      "addc.cc.u64 %1, %1, %11;\n"
      "addc.cc.u64 %2, %2, %12;\n"
      "addc.cc.u64 %3, %3, %13;\n"
      "addc.cc.u64 %4, %4, %14;\n"
      "addc.cc.u64 %5, %5, %15;\n"
      "addc.cc.u64 %6, %6, %16;\n"
      "addc.cc.u64 %7, %7, %17;\n"
      "addc.cc.u64 %8, %8, %18;\n"
      "addc.u64 %9, %9, %19;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1]), "+l"(T[2]), "+l"(T[3]), "+l"(T[4]), "+l"(T[5]), "+l"(T[6]), "+l"(T[7]), "+l"(T[8]), "+l"(T[9])
      : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(A[7]), "l"(A[8]), "l"(A[9]));
}
template <>
__device__ __forceinline__ void sub_limbs<10>(uint64_t (&T)[10], const uint64_t (&A)[10]) {
  asm("{\n"
      "sub.cc.u64 %0, %0, %10;\n"
      "subc.cc.u64 %1, %1, %11;\n"
      "subc.cc.u64 %2, %2, %12;\n"
      "subc.cc.u64 %3, %3, %13;\n"
      "subc.cc.u64 %4, %4, %14;\n"
      "subc.cc.u64 %5, %5, %15;\n"
      "subc.cc.u64 %6, %6, %16;\n"
      "subc.cc.u64 %7, %7, %17;\n"
      "subc.cc.u64 %8, %8, %18;\n"
      "subc.u64 %9, %9, %19;\n"
      "}"
      : "+l"(T[0]), "+l"(T[1]), "+l"(T[2]), "+l"(T[3]), "+l"(T[4]), "+l"(T[5]), "+l"(T[6]), "+l"(T[7]), "+l"(T[8]), "+l"(T[9])
      : "l"(A[0]), "l"(A[1]), "l"(A[2]), "l"(A[3]), "l"(A[4]), "l"(A[5]), "l"(A[6]), "l"(A[7]), "l"(A[8]), "l"(A[9]));
}
#endif

// Fixed-point value of one entry in NL limbs (two's complement, little endian):
// T = sum_j trunc(x_j 2^F), every word's truncated magnitude (a 53-bit integer
// shifted to limbs li, li+1) added or subtracted with one carry chain.
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
    uint64_t A[NL];
#pragma unroll
    for (int i = 0; i < NL; ++i) A[i] = (i == li) ? lo : ((i == li + 1) ? hi : 0);
    if (neg) sub_limbs<NL>(T, A);
    else add_limbs<NL>(T, A);
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
  return __ushort_as_bfloat16(small_int_bf16(d));  // |d| <= 2^(w-1) <= 256: exact
}
template <>
__device__ __forceinline__ double to_out<double>(int d) { return (double)d; }

template <typename Out>
__device__ __forceinline__ void store2(Out *p, int d0, int d1);
template <>
__device__ __forceinline__ void store2<__nv_bfloat16>(__nv_bfloat16 *p, int d0, int d1) {
  *reinterpret_cast<uint32_t *>(p) =
      (uint32_t)small_int_bf16(d0) | ((uint32_t)small_int_bf16(d1) << 16);
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

// The same for w = 8, digits from the bytes of T + H (see cut_one_w8).
template <int NL>
__device__ __forceinline__ bool in_range_w8(const uint64_t (&T)[NL], int S);
template <int NL>
__device__ __forceinline__ bool add_bias_w8(uint64_t (&T)[NL], int S);

template <int MW, int NL, typename Out>
__device__ __forceinline__ void cut_pair_w8(const double (&w0)[MW], const double (&w1)[MW], int F,
                                            int S, Out *dst, int64_t plane, unsigned int *status) {
  uint64_t T0[NL], T1[NL];
  fixed_point<MW, NL>(w0, F, T0);
  fixed_point<MW, NL>(w1, F, T1);
  if (!(in_range_w8<NL>(T0, S) && in_range_w8<NL>(T1, S))) raise_status(status, MW_ERANGE);
  const bool n0 = add_bias_w8<NL>(T0, S), n1 = add_bias_w8<NL>(T1, S);
  Out *q = dst + (int64_t)(S - 1) * plane;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * i + j;
      const int u0 = (int)((T0[i] >> (8 * j)) & 0xFF), u1 = (int)((T1[i] >> (8 * j)) & 0xFF);
      if (k < S - 1) {
        store2<Out>(q, u0 - 128, u1 - 128);
        q -= plane;
      } else if (k == S - 1) {
        store2<Out>(q, n0 ? u0 - 256 : u0, n1 ? u1 - 256 : u1);
      }
    }
  }
}

// One entry, any w: the digits least significant first with a carry.
template <int MW, int NL, typename Out>
__device__ __forceinline__ void cut_one(const double (&x)[MW], int F, int w, int S, Out *dst,
                                        int64_t plane, unsigned int *status) {
  uint64_t T[NL];
  fixed_point<MW, NL>(x, F, T);
  const uint64_t mask = (1ull << w) - 1;
  const int half = 1 << (w - 1);
  int c = 0;
  Out *q = dst + (int64_t)(S - 1) * plane;
  for (int p = S - 1; p >= 1; --p, q -= plane) {
    int r = (int)(T[0] & mask) + c;
    c = r >= half;
    r -= c << w;
    *q = to_out<Out>(r);
    shr<NL>(T, w);
  }
  bool ok = true;
  const int64_t t0 = (int64_t)T[0];
#pragma unroll
  for (int i = 1; i < NL; ++i) ok &= T[i] == (uint64_t)(t0 >> 63);
  ok &= t0 >= -half && t0 < half;
  if (!ok) raise_status(status, MW_ERANGE);
  *dst = to_out<Out>((int)t0 + c);
}

// One entry, w = 8.  Balanced digits d_k in [-128, 128) for k < S-1 are the
// bytes of T + H minus 128, H = 128 (1 + 2^8 + ... + 2^(8(S-2))): adding 128 to
// every low digit maps [-128, 128) onto the byte range, so no carry links the
// digits.  The top digit is (T + H) >> 8(S-1), in [-128, 128] when T lies in
// [-2^(8S-1), 2^(8S-1)) (checked on T first).
template <int NL>
__device__ __forceinline__ bool in_range_w8(const uint64_t (&T)[NL], int S) {
  // the bits of T from 8S-1 up are all equal
  const int b = 8 * S - 1, lb = b >> 6, ob = b & 63;
  int64_t v = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i)
    if (i == lb) v = (int64_t)T[i] >> ob;
  bool ok = v == 0 || v == -1;
#pragma unroll
  for (int i = 0; i < NL; ++i)
    if (i > lb) ok &= T[i] == (uint64_t)v;
  return ok;
}

// T += H = 128 (1 + 2^8 + ... + 2^(8(S-2))); returns the sign of the sum.
template <int NL>
__device__ __forceinline__ bool add_bias_w8(uint64_t (&T)[NL], int S) {
  uint64_t carry = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const int nb = min(max(S - 1 - 8 * i, 0), 8);          // biased bytes in limb i
    const uint64_t h = nb == 8 ? 0x8080808080808080ull
                               : (0x8080808080808080ull & ((1ull << (8 * nb)) - 1));
    const uint64_t s1 = T[i] + h;
    const uint64_t c1 = s1 < h;
    const uint64_t s2 = s1 + carry;
    carry = c1 | (s2 < carry);
    T[i] = s2;
  }
  return (int64_t)T[NL - 1] < 0;
}

// One entry, w = 8.  Balanced digits d_k in [-128, 128) for k < S-1 are the
// bytes of T + H minus 128: adding 128 to every low digit maps [-128, 128)
// onto the byte range, so no carry links the digits.  The top digit is
// (T + H) >> 8(S-1), in [-128, 128] when T lies in [-2^(8S-1), 2^(8S-1))
// (checked on T first): byte S-1, less 256 when the sum is negative.
template <int MW, int NL, typename Out>
__device__ __forceinline__ void cut_one_w8(const double (&x)[MW], int F, int S, Out *dst,
                                           int64_t plane, unsigned int *status) {
  uint64_t T[NL];
  fixed_point<MW, NL>(x, F, T);
  if (!in_range_w8<NL>(T, S)) raise_status(status, MW_ERANGE);
  const bool neg = add_bias_w8<NL>(T, S);
  Out *q = dst + (int64_t)(S - 1) * plane;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = 8 * i + j;
      const int u = (int)((T[i] >> (8 * j)) & 0xFF);
      if (k < S - 1) {
        *q = to_out<Out>(u - 128);
        q -= plane;
      } else if (k == S - 1) {
        *q = to_out<Out>(neg ? u - 256 : u);
      }
    }
  }
}

}  // namespace
}  // namespace mw
