// Cutting entries into pieces and rounding exact integers into m words with a
// per-thread column of 32-bit words in shared memory, indexed at run time, so
// that each word of an m-double touches only the few slots or limbs at its own
// position (device side; also compiles as plain C++).
//   cut_column:   the balanced w-bit digits (w = 8 or 24) of
//                 T = sum_j trunc(x_j 2^F) (Section 2's pieces on the shared
//                 grid): each word adds its truncated magnitude as four signed
//                 24-bit fields into the slots it covers, then one carry pass
//                 from the least significant slot yields the digits;
//   round_column: the m nonoverlapping doubles of X 2^ex, each the value
//                 rounded to nearest (ties to even) of what the previous words
//                 left over (Section 4's final renormalisation, greedy), read
//                 from the two's complement limbs of X without rewriting them.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define MW_HD __host__ __device__ __forceinline__
#else
#define MW_HD inline
#endif

namespace mw {
namespace {

MW_HD uint64_t col_bits(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}
MW_HD double col_double(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
#endif
}
MW_HD int col_clz(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __clz(x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}
MW_HD int col_ctz(uint32_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __ffs((int)x) - 1;
#else
  return __builtin_ctz(x);
#endif
}

MW_HD uint32_t col_fshl(uint32_t lo, uint32_t hi, int n) {  // high word of (hi:lo) << n, n < 32
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, n);
#else
  return (uint32_t)(((((uint64_t)hi << 32) | lo) << n) >> 32);
#endif
}
MW_HD uint32_t col_fshr(uint32_t lo, uint32_t hi, int n) {  // low word of (hi:lo) >> n, n < 32
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(lo, hi, n);
#else
  return (uint32_t)((((uint64_t)hi << 32) | lo) >> n);
#endif
}
MW_HD float col_float(uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, sizeof f);
  return f;
#endif
}
MW_HD uint32_t col_fbits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  uint32_t b;
  std::memcpy(&b, &f, sizeof b);
  return b;
#endif
}

// bfloat16 bits of an integer |d| <= 2^8 (exact): 1.5 2^23 + d has the float
// bit pattern 0x4B400000 + d, less 1.5 2^23 it is d; a float of at most 8
// significant bits is its top 16 bits.
MW_HD uint16_t small_int_bf16(int32_t d) {
  return (uint16_t)(col_fbits(col_float(0x4B400000u + (uint32_t)d) - 12582912.0f) >> 16);
}

// Slots of the column for S digits of w bits: the 24-bit chunk holding the top
// digit, Ct = w (S-1) / 24, the ones below it and three above it (the highest
// a word's four fields can reach; they stay zero for in-range input).
MW_HD int cut_column_slots(int w, int S) { return w * (S - 1) / 24 + 4; }

// Balanced digits d_k (k = 0 least significant) of T = sum_j trunc(x_j 2^F):
// d_k in [-2^(w-1), 2^(w-1)) for k < S-1, the top digit d_(S-1) the rest (in
// [-2^(w-1), 2^(w-1)] when T lies in [-2^(wS-1), 2^(wS-1))).  emit(k, d) is
// called once per digit in the order k = 0, 1, ..., S-1.  Returns false when T
// lies outside that range.
// col: this thread's column, slot c at col[c * stride], cut_column_slots(w, S)
// of them, all zero on entry and left zero.  Slot c collects bits 24c .. 24c+23
// of every word plus a signed excess; the carry pass adds the bias
// H = 2^(w-1) (1 + 2^w + ... + 2^(w(S-2))), after which every digit below the
// top one is a plain w-bit field minus 2^(w-1).
template <int MW, int W, class Emit>
MW_HD bool cut_column(const double (&x)[MW], int F, int S, uint32_t *col, int stride, Emit emit) {
  static_assert(W == 8 || W == 24, "digit widths 8 and 24");
  constexpr int32_t kHalf = 1 << (W - 1);
  constexpr int32_t kBias = W == 24 ? kHalf : 0x808080;   // H restricted to a full chunk
  const int Ct = W * (S - 1) / 24;
#pragma unroll
  for (int j = 0; j < MW; ++j) {
    const uint64_t b = col_bits(x[j]);
    const uint32_t bh = (uint32_t)(b >> 32);
    const int be = (int)((bh >> 20) & 0x7ff);
    const uint32_t mlo = (uint32_t)b;
    const uint32_t mhi = (bh & 0xFFFFFu) | (be ? 0x100000u : 0u);   // M = mhi:mlo < 2^53
    const int sh = (be ? be : 1) - 1075 + F;      // weight of M's last bit on the grid
    // y = trunc(M 2^min(sh, 0)) at bit pos = max(sh, 0)
    uint32_t ylo = mlo, yhi = mhi;
    int pos = sh;
    if (sh < 0) {
      const int r = -sh;
      ylo = r < 32 ? col_fshr(mlo, mhi, r) : (r < 64 ? mhi >> (r - 32) : 0u);
      yhi = r < 32 ? mhi >> r : 0u;
      pos = 0;
    }
    if (pos >= 24 * (Ct + 1)) {                     // only words the exponent does not cover
      ylo = yhi = 0;                                // (non-finite input, flagged elsewhere)
      pos = 0;
    }
    const int c = pos / 24, o = pos - 24 * c;
    const uint32_t w0 = ylo << o, w1 = col_fshl(ylo, yhi, o), w2 = col_fshl(yhi, 0u, o);
    const int32_t f0 = (int32_t)(w0 & 0xFFFFFFu);
    const int32_t f1 = (int32_t)(col_fshr(w0, w1, 24) & 0xFFFFFFu);
    const int32_t f2 = (int32_t)(col_fshr(w1, w2, 16) & 0xFFFFFFu);
    const int32_t f3 = (int32_t)(w2 >> 8);
    const int32_t s = (bh >> 31) ? -1 : 1;
    uint32_t *p = col + c * stride;
    p[0] = (uint32_t)((int32_t)p[0] + s * f0);
    p[stride] = (uint32_t)((int32_t)p[stride] + s * f1);
    p[2 * stride] = (uint32_t)((int32_t)p[2 * stride] + s * f2);
    p[3 * stride] = (uint32_t)((int32_t)p[3 * stride] + s * f3);
  }
  // carry pass; lsign: sign of the digits below the current chunk's, read off
  // the most significant nonzero digit (balanced digits), one compare a chunk
  int32_t carry = 0;
  int lsign = 0;
#pragma unroll
  for (int c = 0; c < Ct; ++c) {
    const int32_t v = (int32_t)col[c * stride] + carry + kBias;
    col[c * stride] = 0u;
    carry = v >> 24;
    const int32_t u = v & 0xFFFFFF;
    if (u != kBias) lsign = u > kBias ? 1 : -1;
    if (W == 24) {
      emit(c, u - kHalf);
    } else {
      emit(3 * c, (u & 0xFF) - 128);
      emit(3 * c + 1, ((u >> 8) & 0xFF) - 128);
      emit(3 * c + 2, (u >> 16) - 128);
    }
  }
  const int nb = W == 24 ? 0 : S - 1 - 3 * Ct;     // digits of chunk Ct below the top one
  const int32_t v = (int32_t)col[Ct * stride] + carry + (W == 24 ? 0 : (0x808080 & ((1 << (8 * nb)) - 1)));
  for (int i = 0; i < nb; ++i) {
    const int32_t d = ((v >> (8 * i)) & 0xFF) - 128;
    emit(3 * Ct + i, d);
    if (d != 0) lsign = d > 0 ? 1 : -1;
  }
  const int32_t top = v >> (W == 24 ? 0 : 8 * nb);
  emit(S - 1, top);
  const uint32_t above = col[(Ct + 1) * stride] | col[(Ct + 2) * stride] | col[(Ct + 3) * stride];
  col[Ct * stride] = 0u;
  col[(Ct + 1) * stride] = 0u;
  col[(Ct + 2) * stride] = 0u;
  col[(Ct + 3) * stride] = 0u;
  // T = top 2^(w(S-1)) + L, |L| < 2^(w(S-1)), L of sign lsign: in range for
  // |top| < 2^(w-1), for top = -2^(w-1) with L >= 0 and top = 2^(w-1) with L < 0
  return above == 0u && ((top > -kHalf && top < kHalf) || (top == -kHalf && lsign >= 0) ||
                         (top == kHalf && lsign < 0));
}

// X 2^ex into MW words by greedy rounding to nearest, ties to even: word k is
// the remainder left by words 0 .. k-1 rounded to 53 bits; zeros once the
// remainder vanishes.  U: X in NL32 32-bit limbs, two's complement.  col: this
// thread's column of NL32 words (limb L at col[L * stride]).
// The remainder below the last cut is never written back: with l the lowest
// set bit of X, the magnitude of -X and of each remainder after a word that
// rounded up is X's own bits inverted above l and kept at and below l (the
// negation of a two's complement integer), so one flag, flipped at every
// rounding up, says which of the two readings applies, and the bits below any
// window are nonzero exactly when l lies below it.
template <int MW, int NL32, class Store>
MW_HD void round_column(const uint32_t (&U)[NL32], uint32_t *col, int stride, int ex,
                        Store store) {
  int lw = -1;
  uint32_t lv = 0;
#pragma unroll
  for (int i = NL32 - 1; i >= 0; --i) {
    col[i * stride] = U[i];
    if (U[i] != 0) {
      lw = i;
      lv = U[i];
    }
  }
  int k = 0;
  if (lw >= 0) {
    const int ell = 32 * lw + col_ctz(lv);
    const uint32_t inv_l = ~((2u << (ell & 31)) - 1u);    // bits above l in limb lw
    bool flip = (int32_t)U[NL32 - 1] < 0;                 // reading: inverted above l
    bool neg = flip;
    int cutp = 32 * NL32;                                 // bits at and above are cleared
#pragma unroll 1
    for (; k < MW && ell < cutp; ++k) {
      const int Lc = cutp >> 5;
      const uint32_t cm = (1u << (cutp & 31)) - 1u;
      auto limb = [&](int L) -> uint32_t {
        if (L < 0) return 0u;
        uint32_t v = col[L * stride];
        if (flip) v ^= L > lw ? 0xFFFFFFFFu : (L == lw ? inv_l : 0u);
        return L < Lc ? v : (L == Lc ? (v & cm) : 0u);
      };
      int h = (cutp - 1) >> 5;
      uint32_t a = limb(h);
      while (a == 0 && h > lw) a = limb(--h);           // bit l is set: ends at lw at the latest
      const uint32_t b = limb(h - 1), c = limb(h - 2);
      const bool below = ell < 32 * (h - 2);
      const int lz = col_clz(a);
      const uint64_t ab = ((uint64_t)a << 32) | b;
      const uint64_t top = lz ? (ab << lz) | (c >> (32 - lz)) : ab;
      const uint32_t c_low = c << lz;                     // bits of c below the window
      uint64_t mant = top >> 11;
      const uint32_t rbit = (uint32_t)(top >> 10) & 1u;
      const bool sticky = ((top & 0x3FF) | c_low) != 0 || below;
      const uint32_t up = rbit & (uint32_t)(sticky | (mant & 1));
      mant += up;
      const int cut = 32 * h - 21 - lz;                   // weight of the mantissa's last bit
      const int e = ex + cut;
      const int bexp = e + 52 + 1023;                     // mant in [2^52, 2^53]
      double mag;
      if (bexp >= 1 && bexp <= 2045)
        mag = col_double(((uint64_t)bexp << 52) + (mant - (1ull << 52)));
      else
        mag = scalbn((double)mant, e);
      store(k, neg ? -mag : mag);
      if (up) {
        flip = !flip;
        neg = !neg;
      }
      cutp = cut;
    }
  }
  for (; k < MW; ++k) store(k, 0.0);
}

}  // namespace
}  // namespace mw
