// Exact fusion of the partial sums and rounding to m words (device side,
// shared by the single and batched combine kernels).
//   add_shifted:    X += V 2^sh on an NL-limb (64-bit) two's complement integer;
//   fuse_diagonals: X += sum_t s_t 2^(w (D-1-t)), any w, 64-bit limbs;
//   fuse_w8:        the same sum for w = 8 straight into 32-bit limbs;
//   round_words32:  the m nonoverlapping doubles of X 2^ex, each the value
//                   rounded to nearest (ties to even) of what the previous
//                   words left over (greedy), computed on the exact integer.
#pragma once
#include <cstdint>

namespace mw {
namespace {

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

// X += sum_t s_t 2^(w (D-1-t)) for the int32 diagonal sums s_t = p[t * plane]
// (any w): 8 independent loads at a time, then Horner in int64 over each group
// of `group` consecutive diagonals (exact for the planner's group size) and one
// multi-limb add per group.
template <int NL>
__device__ __forceinline__ void fuse_diagonals(uint64_t (&X)[NL], const int32_t *p, int64_t plane,
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
__device__ __forceinline__ void to_limbs32(const uint64_t (&X)[NL], uint32_t (&U)[2 * NL]) {
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
// plus the signed carry out of limb j-1.
template <int NL32>
__device__ __forceinline__ void fuse_w8(uint32_t (&U)[NL32], const int32_t *p, int64_t plane,
                                        int D) {
  static_assert(NL32 % 2 == 0, "limbs in pairs");
  const int32_t *last = p + (int64_t)(D - 1) * plane;   // s_{D-1}, weight 2^0
  int64_t R = 0;
#pragma unroll
  for (int j = 0; j < NL32; j += 2) {
    int32_t s[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int u = 4 * j + k;                            // s_{D-1-u}, weight 2^(8u)
      s[k] = u < D ? last[-(int64_t)u * plane] : 0;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
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

// N = -U (two's complement) on NL32 32-bit limbs: one sub.cc/subc borrow chain
// on the device (the loop below is the same arithmetic for other compilers).
template <int NL32>
__device__ __forceinline__ void neg_limbs32(const uint32_t (&U)[NL32], uint32_t (&N)[NL32]) {
  uint32_t c = 1;
#pragma unroll
  for (int i = 0; i < NL32; ++i) {
    N[i] = ~U[i] + c;
    c &= (uint32_t)(N[i] == 0);
  }
}
#if defined(__CUDA_ARCH__)
template <>
__device__ __forceinline__ void neg_limbs32<8>(const uint32_t (&U)[8], uint32_t (&N)[8]) {
  asm("{\n"
      "sub.cc.u32 %0, 0, %8;\n"
      "subc.cc.u32 %1, 0, %9;\n"
      "subc.cc.u32 %2, 0, %10;\n"
      "subc.cc.u32 %3, 0, %11;\n"
      "subc.cc.u32 %4, 0, %12;\n"
      "subc.cc.u32 %5, 0, %13;\n"
      "subc.cc.u32 %6, 0, %14;\n"
      "subc.u32 %7, 0, %15;\n"
      "}"
      : "=r"(N[0]), "=r"(N[1]), "=r"(N[2]), "=r"(N[3]), "=r"(N[4]), "=r"(N[5]), "=r"(N[6]), "=r"(N[7])
      : "r"(U[0]), "r"(U[1]), "r"(U[2]), "r"(U[3]), "r"(U[4]), "r"(U[5]), "r"(U[6]), "r"(U[7]));
}
template <>
__device__ __forceinline__ void neg_limbs32<10>(const uint32_t (&U)[10], uint32_t (&N)[10]) {
  asm("{\n"
      "sub.cc.u32 %0, 0, %10;\n"
      "subc.cc.u32 %1, 0, %11;\n"
      "subc.cc.u32 %2, 0, %12;\n"
      "subc.cc.u32 %3, 0, %13;\n"
      "subc.cc.u32 %4, 0, %14;\n"
      "subc.cc.u32 %5, 0, %15;\n"
      "subc.cc.u32 %6, 0, %16;\n"
      "subc.cc.u32 %7, 0, %17;\n"
      "subc.cc.u32 %8, 0, %18;\n"
      "subc.u32 %9, 0, %19;\n"
      "}"
      : "=r"(N[0]), "=r"(N[1]), "=r"(N[2]), "=r"(N[3]), "=r"(N[4]), "=r"(N[5]), "=r"(N[6]), "=r"(N[7]), "=r"(N[8]), "=r"(N[9])
      : "r"(U[0]), "r"(U[1]), "r"(U[2]), "r"(U[3]), "r"(U[4]), "r"(U[5]), "r"(U[6]), "r"(U[7]), "r"(U[8]), "r"(U[9]));
}
template <>
__device__ __forceinline__ void neg_limbs32<12>(const uint32_t (&U)[12], uint32_t (&N)[12]) {
  asm("{\n"
      "sub.cc.u32 %0, 0, %12;\n"
      "subc.cc.u32 %1, 0, %13;\n"
      "subc.cc.u32 %2, 0, %14;\n"
      "subc.cc.u32 %3, 0, %15;\n"
      "subc.cc.u32 %4, 0, %16;\n"
      "subc.cc.u32 %5, 0, %17;\n"
      "subc.cc.u32 %6, 0, %18;\n"
      "subc.cc.u32 %7, 0, %19;\n"
      "subc.cc.u32 %8, 0, %20;\n"
      "subc.cc.u32 %9, 0, %21;\n"
      "subc.cc.u32 %10, 0, %22;\n"
      "subc.u32 %11, 0, %23;\n"
      "}"
      : "=r"(N[0]), "=r"(N[1]), "=r"(N[2]), "=r"(N[3]), "=r"(N[4]), "=r"(N[5]), "=r"(N[6]), "=r"(N[7]), "=r"(N[8]), "=r"(N[9]), "=r"(N[10]), "=r"(N[11])
      : "r"(U[0]), "r"(U[1]), "r"(U[2]), "r"(U[3]), "r"(U[4]), "r"(U[5]), "r"(U[6]), "r"(U[7]), "r"(U[8]), "r"(U[9]), "r"(U[10]), "r"(U[11]));
}
template <>
__device__ __forceinline__ void neg_limbs32<14>(const uint32_t (&U)[14], uint32_t (&N)[14]) {
  asm("{\n"
      "sub.cc.u32 %0, 0, %14;\n"
      "subc.cc.u32 %1, 0, %15;\n"
      "subc.cc.u32 %2, 0, %16;\n"
      "subc.cc.u32 %3, 0, %17;\n"
      "subc.cc.u32 %4, 0, %18;\n"
      "subc.cc.u32 %5, 0, %19;\n"
      "subc.cc.u32 %6, 0, %20;\n"
      "subc.cc.u32 %7, 0, %21;\n"
      "subc.cc.u32 %8, 0, %22;\n"
      "subc.cc.u32 %9, 0, %23;\n"
      "subc.cc.u32 %10, 0, %24;\n"
      "subc.cc.u32 %11, 0, %25;\n"
      "subc.cc.u32 %12, 0, %26;\n"
      "subc.u32 %13, 0, %27;\n"
      "}"
      : "=r"(N[0]), "=r"(N[1]), "=r"(N[2]), "=r"(N[3]), "=r"(N[4]), "=r"(N[5]), "=r"(N[6]), "=r"(N[7]), "=r"(N[8]), "=r"(N[9]), "=r"(N[10]), "=r"(N[11]), "=r"(N[12]), "=r"(N[13])
      : "r"(U[0]), "r"(U[1]), "r"(U[2]), "r"(U[3]), "r"(U[4]), "r"(U[5]), "r"(U[6]), "r"(U[7]), "r"(U[8]), "r"(U[9]), "r"(U[10]), "r"(U[11]), "r"(U[12]), "r"(U[13]));
}
template <>
__device__ __forceinline__ void neg_limbs32<16>(const uint32_t (&U)[16], uint32_t (&N)[16]) {
  asm("{\n"
      "sub.cc.u32 %0, 0, %16;\n"
      "subc.cc.u32 %1, 0, %17;\n"
      "subc.cc.u32 %2, 0, %18;\n"
      "subc.cc.u32 %3, 0, %19;\n"
      "subc.cc.u32 %4, 0, %20;\n"
      "subc.cc.u32 %5, 0, %21;\n"
      "subc.cc.u32 %6, 0, %22;\n"
      "subc.cc.u32 %7, 0, %23;\n"
      "subc.cc.u32 %8, 0, %24;\n"
      "subc.cc.u32 %9, 0, %25;\n"
      "subc.cc.u32 %10, 0, %26;\n"
      "subc.cc.u32 %11, 0, %27;\n"
      "subc.cc.u32 %12, 0, %28;\n"
      "subc.cc.u32 %13, 0, %29;\n"
      "subc.cc.u32 %14, 0, %30;\n"
      "subc.u32 %15, 0, %31;\n"
      "}"
      : "=r"(N[0]), "=r"(N[1]), "=r"(N[2]), "=r"(N[3]), "=r"(N[4]), "=r"(N[5]), "=r"(N[6]), "=r"(N[7]), "=r"(N[8]), "=r"(N[9]), "=r"(N[10]), "=r"(N[11]), "=r"(N[12]), "=r"(N[13]), "=r"(N[14]), "=r"(N[15])
      : "r"(U[0]), "r"(U[1]), "r"(U[2]), "r"(U[3]), "r"(U[4]), "r"(U[5]), "r"(U[6]), "r"(U[7]), "r"(U[8]), "r"(U[9]), "r"(U[10]), "r"(U[11]), "r"(U[12]), "r"(U[13]), "r"(U[14]), "r"(U[15]));
}
template <>
__device__ __forceinline__ void neg_limbs32<18>(const uint32_t (&U)[18], uint32_t (&N)[18]) {
  asm("{\n"
      "sub.cc.u32 %0, 0, %18;\n"
      "subc.cc.u32 %1, 0, %19;\n"
      "subc.cc.u32 %2, 0, %20;\n"
      "subc.cc.u32 %3, 0, %21;\n"
      "subc.cc.u32 %4, 0, %22;\n"
      "subc.cc.u32 %5, 0, %23;\n"
      "subc.cc.u32 %6, 0, %24;\n"
      "subc.cc.u32 %7, 0, %25;\n"
      "subc.cc.u32 %8, 0, %26;\n"
      "subc.cc.u32 %9, 0, %27;\n"
      "subc.cc.u32 %10, 0, %28;\n"
      "subc.cc.u32 %11, 0, %29;\n"
      "subc.cc.u32 %12, 0, %30;\n"
      "subc.cc.u32 %13, 0, %31;\n"
      "subc.cc.u32 %14, 0, %32;\n"
      "subc.cc.u32 %15, 0, %33;\n"
      "subc.cc.u32 %16, 0, %34;\n"
      "subc.u32 %17, 0, %35;\n"
      "}"
      : "=r"(N[0]), "=r"(N[1]), "=r"(N[2]), "=r"(N[3]), "=r"(N[4]), "=r"(N[5]), "=r"(N[6]), "=r"(N[7]), "=r"(N[8]), "=r"(N[9]), "=r"(N[10]), "=r"(N[11]), "=r"(N[12]), "=r"(N[13]), "=r"(N[14]), "=r"(N[15]), "=r"(N[16]), "=r"(N[17])
      : "r"(U[0]), "r"(U[1]), "r"(U[2]), "r"(U[3]), "r"(U[4]), "r"(U[5]), "r"(U[6]), "r"(U[7]), "r"(U[8]), "r"(U[9]), "r"(U[10]), "r"(U[11]), "r"(U[12]), "r"(U[13]), "r"(U[14]), "r"(U[15]), "r"(U[16]), "r"(U[17]));
}
template <>
__device__ __forceinline__ void neg_limbs32<20>(const uint32_t (&U)[20], uint32_t (&N)[20]) {
  asm("{\n"
      "sub.cc.u32 %0, 0, %20;\n"
      "subc.cc.u32 %1, 0, %21;\n"
      "subc.cc.u32 %2, 0, %22;\n"
      "subc.cc.u32 %3, 0, %23;\n"
      "subc.cc.u32 %4, 0, %24;\n"
      "subc.cc.u32 %5, 0, %25;\n"
      "subc.cc.u32 %6, 0, %26;\n"
      "subc.cc.u32 %7, 0, %27;\n"
      "subc.cc.u32 %8, 0, %28;\n"
      "subc.cc.u32 %9, 0, %29;\n"
      "subc.cc.u32 %10, 0, %30;\n"
      "subc.cc.u32 %11, 0, %31;\n"
      "subc.cc.u32 %12, 0, %32;\n"
      "subc.cc.u32 %13, 0, %33;\n"
      "subc.cc.u32 %14, 0, %34;\n"
      "subc.cc.u32 %15, 0, %35;\n"
      "subc.cc.u32 %16, 0, %36;\n"
      "subc.cc.u32 %17, 0, %37;\n"
      "subc.cc.u32 %18, 0, %38;\n"
      "subc.u32 %19, 0, %39;\n"
      "}"
      : "=r"(N[0]), "=r"(N[1]), "=r"(N[2]), "=r"(N[3]), "=r"(N[4]), "=r"(N[5]), "=r"(N[6]), "=r"(N[7]), "=r"(N[8]), "=r"(N[9]), "=r"(N[10]), "=r"(N[11]), "=r"(N[12]), "=r"(N[13]), "=r"(N[14]), "=r"(N[15]), "=r"(N[16]), "=r"(N[17]), "=r"(N[18]), "=r"(N[19])
      : "r"(U[0]), "r"(U[1]), "r"(U[2]), "r"(U[3]), "r"(U[4]), "r"(U[5]), "r"(U[6]), "r"(U[7]), "r"(U[8]), "r"(U[9]), "r"(U[10]), "r"(U[11]), "r"(U[12]), "r"(U[13]), "r"(U[14]), "r"(U[15]), "r"(U[16]), "r"(U[17]), "r"(U[18]), "r"(U[19]));
}
#endif

// Greedy rounding of X 2^ex, X given as NL32 32-bit limbs (two's complement),
// into MW nonoverlapping doubles: word k is the remainder left by words
// 0..k-1 rounded to nearest (ties to even), all on the exact integer.
// store(k, v) receives word k; words after an exact remainder are zero.
// Per word: find the top nonzero limb h, take a 96-bit window from limbs h,
// h-1, h-2 (53 bits, the rounding bit, the rest sticky with every lower
// limb), then keep the bits below the last mantissa bit (cut), or, rounded up,
// 2^cut minus them (-U mod 2^cut) with the sign flipped.
template <int MW, int NL32, class Store>
__device__ __forceinline__ void round_words32(uint32_t (&U)[NL32], int ex, Store store) {
  bool neg = (int32_t)U[NL32 - 1] < 0;
  if (neg) {
    uint32_t N[NL32];
    neg_limbs32<NL32>(U, N);
#pragma unroll
    for (int i = 0; i < NL32; ++i) U[i] = N[i];
  }
  int k = 0;
#pragma unroll 1
  for (; k < MW; ++k) {
    int h = -1;
#pragma unroll
    for (int i = 0; i < NL32; ++i)
      if (U[i] != 0) h = i;
    if (h < 0) break;
    uint32_t a = 0, b = 0, c = 0, below = 0;
#pragma unroll
    for (int i = 0; i < NL32; ++i) {
      if (i <= h) {
        below |= c;
        c = b;
        b = a;
        a = U[i];
      }
    }
    const int lz = __clz(a);
    const uint64_t ab = ((uint64_t)a << 32) | b;
    const uint64_t top = lz ? (ab << lz) | (c >> (32 - lz)) : ab;
    const uint32_t c_low = c << lz;                       // bits of c below the window
    uint64_t mant = top >> 11;
    const uint32_t rbit = (uint32_t)(top >> 10) & 1u;
    const bool sticky = ((top & 0x3FF) | c_low | below) != 0;
    const uint32_t up = rbit & (uint32_t)(sticky | (mant & 1));
    mant += up;
    const int cut = 32 * h - 21 - lz;                     // weight of the mantissa's last bit
    const double mag = scalbn((double)mant, ex + cut);
    store(k, neg ? -mag : mag);
    // remainder: limbs below the cut limb kept, the cut limb masked, the rest cleared
    const int cl = cut >> 5;                              // negative: everything cleared
    const uint32_t pm = (1u << (cut & 31)) - 1u;
    uint32_t N[NL32];
    neg_limbs32<NL32>(U, N);
#pragma unroll
    for (int i = 0; i < NL32; ++i) {
      const uint32_t x = up ? N[i] : U[i];
      U[i] = i < cl ? x : (i == cl ? (x & pm) : 0u);
    }
    if (up) neg = !neg;
  }
  for (; k < MW; ++k) store(k, 0.0);
}

}  // namespace
}  // namespace mw
