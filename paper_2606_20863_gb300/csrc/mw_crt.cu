// MW_CRT: the residue form of the product (the second Ozaki scheme, which
// Sections 1 and 4 point to as the tensor-core route for the error-free
// summation).
//
// Steps 1-2 stay those of Section 2: one shared exponent per row of op(A) and
// column of op(B), every word truncated on the fixed-point grid of L bits,
//   T = sum_j trunc(x_j 2^(L - 2 - E)),   -2^(L-1) <= T < 2^(L-1).
// Instead of cutting T into w-bit digits and multiplying every pair of digit
// matrices, T is reduced modulo n small pairwise coprime moduli p_i (balanced
// residues, at most floor(p_i / 2) <= 256 in magnitude, so exact in bfloat16),
// and one tensor-core product per modulus gives the exact integer sums
//   Y_i = sum_k r^A_i,k r^B_i,k            (mw_ozaki.cu, its CRT instance).
// The exact product X = sum_k T^A_k T^B_k is the unique integer in (-P/2, P/2]
// with X = Y_i mod p_i, P = p_1 ... p_n > 8 max|X| (Chinese remainder theorem):
//   y_i = Y_i (P/p_i)^(-1) mod p_i,   X = sum_i y_i (P/p_i) - k P,
// k = round(sum_i y_i / p_i), exact because |X| < P/8 leaves the fractional part
// of sum_i y_i / p_i within 1/8 of an integer and the float sum errs by far
// less.  X 2^(E_A + E_B + 4 - L_A - L_B) is rounded into m words greedily
// (round_column), as in the slice form.
//
// This file holds the table of moduli, the residue split and the
// reconstruction; the product kernel is the slice form's, one pair per modulus.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "mw_column.cuh"
#include "mw_device.cuh"
#include "mw_internal.h"
#include "mw_pieces.cuh"
#include "mw_tc.cuh"

namespace mw {
namespace {

// Pairwise coprime odd moduli, at most 513 (balanced residues within
// bfloat16's exact integers; odd, so that no sum lies halfway between two
// multiples of a modulus and the rounding of z / p below needs no correction).
// An fp32 sum of `chunk` products of residues stays exact below 2^24 when
// chunk floor(p/2)^2 <= 2^24: 4096 products for p <= 129, 2048 for p <= 181,
// 1024 for p <= 257, 512 for p <= 363, 256 for p <= 513.  A modulus costs the
// tensor cores one product of residue matrices, 64-wide k-blocks at about 625
// cycles a 128 x 256 tile, plus per tile the store of its residues, about 6,900
// cycles, and one drain of the fp32 accumulators every chunk, about 1,200 cycles
// (fitted to measurements on GB300).  The table: greedy by log2(p) / cost at
// K = 4096, each step the best odd number coprime to every one taken; a
// product uses the first n moduli.
constexpr uint16_t kModuli[] = {
    257, 255, 253, 251, 247, 241, 239, 181, 233, 179, 229, 227, 223, 173, 359, 217,
    353, 167, 349, 347, 211, 163, 337, 331, 157, 199, 197, 317, 193, 151, 313, 191,
    311, 149, 307, 127, 293, 139, 283, 137, 281, 277, 271, 269, 131, 263, 113, 109,
    107, 103, 101, 97, 509, 503, 499, 491, 487, 479, 89, 467, 463, 461, 457, 449,
    443, 439, 83, 433, 431, 421, 419, 409, 79, 401, 397, 389, 383, 379, 373, 367,
    73, 71, 67, 61, 59, 53, 47, 43, 41, 37, 29};
constexpr int kNumModuli = sizeof(kModuli) / sizeof(kModuli[0]);
static_assert(kNumModuli <= kCrtMaxModuli, "moduli table too long");
constexpr bool all_odd() {
  for (int i = 0; i < kNumModuli; ++i)
    if (kModuli[i] % 2 == 0 || kModuli[i] > 513) return false;
  return true;
}
static_assert(all_odd(), "the moduli must be odd and at most 513");
constexpr int kPow16 = 65;   // 2^(16 j) mod p for j = 0..64 (T of up to 16 64-bit limbs)

// Per modulus: p, floor(2^32 / p) for reducing 32-bit values, p and 1/p in
// float (table entries, so that no conversion instruction runs per residue),
// and 2^(16 j) mod p.
struct CrtTab {
  uint32_t p[kCrtMaxModuli];
  uint32_t m32[kCrtMaxModuli];
  float pf[kCrtMaxModuli], rcp[kCrtMaxModuli];
  uint32_t pow16[kCrtMaxModuli][kPow16];
};
constexpr CrtTab make_crt_tab() {
  CrtTab t{};
  for (int i = 0; i < kNumModuli; ++i) {
    const uint32_t p = kModuli[i];
    t.p[i] = p;
    t.m32[i] = (uint32_t)((1ull << 32) / p);
    t.pf[i] = (float)p;
    t.rcp[i] = 1.0f / (float)p;
    uint32_t x = 1u % p;
    for (int j = 0; j < kPow16; ++j) {
      t.pow16[i][j] = x;
      x = (uint32_t)((uint64_t)x * 65536u % p);
    }
  }
  return t;
}
__constant__ CrtTab kCrt = make_crt_tab();

// x mod p for any 32-bit x: q = floor(x m32 / 2^32) is floor(x/p) or one less.
__device__ __forceinline__ uint32_t mod_u32(uint32_t x, uint32_t p, uint32_t m32) {
  uint32_t r = x - __umulhi(x, m32) * p;
  return r >= p ? r - p : r;
}

// The residue of T in [-floor(p/2), ceil(p/2) - 1]: r >= p - floor(p/2) maps to r - p.
__device__ __forceinline__ int balanced(uint32_t r, uint32_t p) {
  return r >= p - (p >> 1) ? (int)r - (int)p : (int)r;
}

// The balanced residue of an exactly represented float integer z (|z| < 2^22)
// modulo an odd p, in [-floor(p/2), floor(p/2)]: z - q p with q the nearest
// integer to z / p.  fmaf(z, 1/p, 1.5 2^23) rounds the exact product z fl(1/p)
// to an integer; that product differs from z / p by less than |z| 2^-24 / p <
// 1 / (4p), while an integer z over an odd p lies at least 1 / (2p) from any
// half integer, so q is the nearest integer to z / p itself.  Every step is
// exact (|q p| < 2^23).
__device__ __forceinline__ float balanced_f(float z, int t) {
  const float q = fmaf(z, kCrt.rcp[t], 12582912.0f) - 12582912.0f;
  return fmaf(-q, kCrt.pf[t], z);
}

// bfloat16 bits of an integer-valued float of magnitude at most 256 (at most 8
// significant bits): its top 16 bits.
__device__ __forceinline__ uint16_t bf16_bits_small(float r) {
  return (uint16_t)(__float_as_uint(r) >> 16);
}

// T in [-2^(L-1), 2^(L-1)): every bit from L-1 up equals the sign.
template <int NL>
__device__ __forceinline__ bool in_range_bits(const uint64_t (&T)[NL], int L) {
  const int b = L - 1, lb = b >> 6, ob = b & 63;
  int64_t v = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i)
    if (i == lb) v = (int64_t)T[i] >> ob;
  bool ok = (v == 0 || v == -1) && lb < NL;
#pragma unroll
  for (int i = 0; i < NL; ++i)
    if (i > lb) ok &= T[i] == (uint64_t)v;
  return ok;
}

// ---- residue split on the tensor cores -------------------------------------------
// T = sum_q d_q 2^(8q) with balanced base-256 digits d_q (|d| <= 128, the digits
// the slice form cuts with w = 8), so T mod p_t = sum_q d_q c_qt mod p_t with
// c_qt = 2^(8q) mod p_t taken balanced (|c| <= 256).  Two MMAs per tile of 256
// entries (slots 0..255 of the tile's box): A_h (128 x 64) holds the digits of
// the entries in slots 2j + h, in row rho(j) = j ^ ((j >> 4) & 7) (a permutation
// that keeps the threads' shared-memory stores free of bank conflicts), written
// by the threads; B (64 x n) the constants c_qt, built once per CTA, zero for
// q >= S; both in fp16 (exact for integers up to 2048).  The fp32 sums
// |sum_q d_q c_qt| <= 64 2^15 = 2^21 are exact; a thread of the epilogue reads
// the sums of the entries in slots 2j and 2j + 1 (tensor-memory lane rho(j)),
// reduces them mod p_t (balanced_f) and writes both as one pair of bfloat16
// into row t of a shared tile of residues that one TMA store writes to the
// residue planes.
// Digits from bytes: with H = 128 (1 + 2^8 + ... + 2^(8(S-2))), byte q of T + H
// is d_q + 128 for q < S-1; the fp16 number with exponent field 0x64 and that
// byte as low mantissa bits is 1024 + byte, so one byte permute and one packed
// fp16 add of -1152 give two digits.  Every column gets byte - 128, the top
// one too, whose digit is byte S-1 less 256 for a negative T + H: the
// difference, +128 or -128, goes into column 63, whose constants are those of
// column S-1 (S <= 48).  The other columns q >= S multiply zero constants and
// may hold anything finite.
// TRANS = false: a tile is 256 consecutive k of one row r (slot = k); TRANS =
// true (the operand stored K x R): 8 consecutive r x 32 consecutive k (slot =
// 32 r + k), thread i reading r = i mod 8, k = i / 8, so that the loads along r
// fill whole sectors.
constexpr int kResTile = 256;                     // entries of a tile, threads of a CTA
constexpr uint32_t kHalfBytes = 128 * 128;        // one A: 128 rows x 64 fp16

// Bytes of shared memory of the residue split for npad constants rows.
inline size_t residue_smem(int npad) {
  return 1024 + 2 * kHalfBytes + (size_t)npad * 128 + (size_t)npad * 512 + 32;
}
// Tensor-memory columns: two accumulators of npad columns.
__host__ __device__ inline uint32_t residue_tmem_cols(int npad) {
  uint32_t c = 32;
  while (c < 2u * (uint32_t)npad) c *= 2;
  return c;
}
__host__ __device__ __forceinline__ uint32_t res_rho(uint32_t j) { return j ^ ((j >> 4) & 7u); }

template <int MW>
struct SplitEntry {      // one thread's entry of a tile: position and words
  int64_t r, k;
  bool valid;
  double x[MW];
};

template <int MW, int NL, bool TRANS>
__global__ void __launch_bounds__(kResTile, 3)
    residues_mma_kernel(const __grid_constant__ CUtensorMap omap, const double *__restrict__ X,
                        int64_t R, int64_t K, int64_t ld, int64_t ps, int L, int S, int nmod,
                        int npad, int64_t dld, const int *E, unsigned int *status,
                        int32_t *redo, const int32_t *gate) {
  if (gate && *gate == 0) return;                  // the pass over every word is not needed
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sA = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);   // A_0, A_1
  uint8_t *sB = sA + 2 * kHalfBytes;               // npad rows x 64 constants
  uint8_t *stage = sB + (size_t)npad * 128;        // npad rows of 256 residues (512 B)
  uint64_t *bar = (uint64_t *)(stage + (size_t)npad * 512);
  uint32_t *holder = (uint32_t *)(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int idx = tid; idx < npad * 64; idx += kResTile) {
    const int t = idx >> 6, qc = idx & 63;
    const int q = qc == 63 ? S - 1 : qc;       // column 63 repeats the top digit's
    int c = 0;
    if (t < nmod && (q < S || qc == 63)) {
      const uint32_t p = kCrt.p[t];
      uint32_t x = kCrt.pow16[t][q >> 1];
      if (q & 1) x = mod_u32(x * 256u, p, kCrt.m32[t]);
      c = balanced(x, p);
    }
    *reinterpret_cast<uint16_t *>(sB + sw128_offset(t, qc)) = __half_as_ushort(__int2half_rn(c));
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    fence_barrier_init();
    prefetch_map(&omap);
  }
  const uint32_t ncols = residue_tmem_cols(npad);
  if (warp == 0) tmem_alloc(holder, ncols);
  fence_proxy_async_smem();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;
  const uint32_t idesc = idesc_f16(128, npad);
  const int64_t ktiles = TRANS ? (dld + 31) / 32 : (dld + 255) / 256;
  const int64_t rtiles = TRANS ? (R + 7) / 8 : R;
  // tile u = a * inner + b: (rt, kt) = (a, b) for rows (k contiguous), (b, a) for
  // the operand stored K x R, so that the CTAs running together read neighbouring
  // r of the same k rows (whole sectors); each CTA steps u by the grid size
  const int64_t inner = TRANS ? rtiles : ktiles, outer = TRANS ? ktiles : rtiles;
  const int64_t gq = gridDim.x / inner, gr = gridDim.x - gq * inner;
  // this thread's slot in the tile (the box is 256 k of one row, or 8 rows x 32
  // k), and the row of A_(slot & 1) that takes its digits
  const uint32_t slot = TRANS ? (uint32_t)((tid & 7) * 32 + (tid >> 3)) : (uint32_t)tid;
  uint8_t *arow = sA + (slot & 1) * kHalfBytes;
  const uint32_t rowA = res_rho(slot >> 1);
  volatile int abort_flag = 0;

  auto step = [&](int64_t &a, int64_t &b) {
    a += gq;
    b += gr;
    if (b >= inner) {
      b -= inner;
      ++a;
    }
  };
  auto fetch = [&](int64_t ta, int64_t tb, SplitEntry<MW> &e) {
    e.valid = false;
    e.r = e.k = 0;
    if (ta < outer) {
      const int64_t rt = TRANS ? tb : ta, kt = TRANS ? ta : tb;
      e.r = TRANS ? rt * 8 + (tid & 7) : rt;
      e.k = TRANS ? kt * 32 + (tid >> 3) : kt * 256 + tid;
      e.valid = e.r < R && e.k < dld;
    }
    const bool in = e.valid && e.k < K;
#pragma unroll
    for (int j = 0; j < MW; ++j)
      e.x[j] = in ? (TRANS ? X[j * ps + e.k * ld + e.r] : X[j * ps + e.r * ld + e.k]) : 0.0;
  };

  SplitEntry<MW> ec, en;
  uint32_t ph = 0;
  bool ok = true;
  int64_t ca = blockIdx.x / inner, cb = blockIdx.x - (blockIdx.x / inner) * inner;
  fetch(ca, cb, ec);
  for (; ca < outer; step(ca, cb)) {
    // digits of the entry into row tid of A
    {
      uint64_t T[NL];
      fixed_point<MW, NL>(ec.x, ec.valid ? L - 2 - E[ec.r] : 0, T);
      const bool in = in_range_bits<NL>(T, L);
      if (redo) {
        // exponents from the leading words: they hold for this entry when its
        // leading word is normal and no later word has a larger exponent field, or
        // when every word is zero; anything else (and a value out of range) sends
        // the operand through the pass over every word
        const uint32_t e0 = (uint32_t)(__double_as_longlong(ec.x[0]) >> 52) & 0x7ffu;
        bool lead = e0 != 0x7ffu;
        bool rest = false;                         // a later word is nonzero
#pragma unroll
        for (int j = 1; j < MW; ++j) {
          const uint64_t b = (uint64_t)__double_as_longlong(ec.x[j]);
          const uint32_t ej = (uint32_t)(b >> 52) & 0x7ffu;
          lead &= ej <= e0 && ej != 0x7ffu;
          rest |= (b << 1) != 0;
        }
        if (e0 == 0) lead = !rest;                 // zero or subnormal, the only nonzero word
        if (ec.valid && !(lead && in)) atomicExch(redo, 1);
      } else if (ec.valid && !in) {
        raise_status(status, MW_ERANGE);
      }
      const bool neg = add_bias_w8<NL>(T, S);
#pragma unroll
      for (int c = 0; c < 8; ++c) {               // 16-byte chunk c: digits 8c .. 8c+7
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (c < NL) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t word = (uint32_t)(T[c < NL ? c : 0] >> (32 * h));
            uint32_t lo, hi;
            asm("prmt.b32 %0, %1, %2, 0x5140;" : "=r"(lo) : "r"(word), "r"(0x64646464u));
            asm("prmt.b32 %0, %1, %2, 0x7362;" : "=r"(hi) : "r"(word), "r"(0x64646464u));
            asm("add.rn.f16x2 %0, %1, %2;" : "=r"(w[2 * h]) : "r"(lo), "r"(0xE480E480u));
            asm("add.rn.f16x2 %0, %1, %2;" : "=r"(w[2 * h + 1]) : "r"(hi), "r"(0xE480E480u));
          }
        }
        if (c == 7) w[3] = neg ? 0xD8000000u : 0x58000000u;   // column 63: -128 / +128 in fp16
        *reinterpret_cast<uint4 *>(arow + sw128_offset(rowA, 8 * c)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    fence_proxy_async_smem();
    if (tid == 0) bulk_wait_read();                // the previous tile's store has read its tile
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint64_t a0 = sw128_desc(smem_u32(sA)), a1 = sw128_desc(smem_u32(sA + kHalfBytes));
      const uint64_t bd = sw128_desc(smem_u32(sB));
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) tc_mma(tmem, a0 + 2 * kk, bd + 2 * kk, idesc, kk ? 1u : 0u);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        tc_mma(tmem + npad, a1 + 2 * kk, bd + 2 * kk, idesc, kk ? 1u : 0u);
      tc_commit(&bar[0]);
    }
    {
      int64_t na = ca, nb = cb;
      step(na, nb);
      fetch(na, nb, en);                           // the next tile's words load meanwhile
    }
    ok = __syncthreads_and(mbar_wait(&bar[0], ph, status, &abort_flag));
    if (!ok) break;
    ph ^= 1;
    tc_fence_after();
    // every sum reduced mod p_t into row t of the shared tile: warp w reads lanes
    // 32 (w % 4).. (slot pairs rho(lane)) and, of every 32 moduli, the 16 of half
    // w / 4 (compile-time indices, so the constants of balanced_f stay operands)
    {
      const uint32_t lane32 = (uint32_t)((warp & 3) * 32 + (tid & 31));
      const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16);
      uint32_t *dst = reinterpret_cast<uint32_t *>(stage) + res_rho(lane32);
      auto reduce = [&](auto half) {
        constexpr int HF = decltype(half)::value;
#pragma unroll
        for (int h = 0; h < 3; ++h) {
          const int t0 = 32 * h + 16 * HF;
          if (t0 >= nmod) break;
          uint32_t ve[16], vo[16];
          tc_ld16(ta + t0, ve);
          tc_ld16(ta + npad + t0, vo);
          tc_wait_ld();
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            if (t0 + u >= nmod) break;
            const float re = balanced_f(__uint_as_float(ve[u]), 32 * h + 16 * HF + u);
            const float ro = balanced_f(__uint_as_float(vo[u]), 32 * h + 16 * HF + u);
            uint32_t pr;
            asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(pr) : "f"(ro), "f"(re));
            dst[(size_t)(t0 + u) * 128] = pr;
          }
        }
      };
      if (warp < 4) reduce(std::integral_constant<int, 0>());
      else reduce(std::integral_constant<int, 1>());
    }
    tc_fence_before();
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {                                // entries past R or dld are clipped
      if (TRANS) tma_store_3d(&omap, (int)(ca * 32), (int)(cb * 8), 0, smem_u32(stage));
      else tma_store_3d(&omap, (int)(cb * 256), (int)ca, 0, smem_u32(stage));
    }
    ec = en;
  }
  if (!ok && tid == 0) {                           // a wait gave up: let the product finish
    volatile int never = 0;
    mbar_wait(&bar[0], ph, status, &never);
  }
  if (tid == 0) bulk_wait_all();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_free(tmem, ncols);
  }
}

template <int MW, int NL>
int launch_residues_t(const SplitArgs &a, cudaStream_t s) {
  const int S = (a.S + 7) / 8;                     // base-256 digits of an L-bit T
  const int npad = (a.nmod + 15) / 16 * 16;
  if (S > 8 * NL || S > 48 || NL > 6 || npad > 96)
    return fail(MW_EUNSUPPORTED, "residue split: %d digits, %d moduli", S, a.nmod);
  if (a.digit_ld % 8 || a.R > 0x7fffffffLL || a.digit_ld > 0x7fffffffLL)
    return fail(MW_EUNSUPPORTED, "residue split: planes of %lld x %lld", (long long)a.R,
                (long long)a.digit_ld);
  // residue planes [t][r][k] of dld columns; boxes of one row x 256 k, or 8 rows
  // x 32 k, every modulus; no swizzle (the shared tile is dense)
  alignas(64) CUtensorMap map;
  const uint64_t dims[3] = {(uint64_t)a.digit_ld, (uint64_t)a.R, (uint64_t)a.nmod};
  const uint64_t strides[2] = {(uint64_t)a.digit_ld * 2, (uint64_t)a.R * a.digit_ld * 2};
  const uint32_t box[3] = {a.trans ? 32u : 256u, a.trans ? 8u : 1u, (uint32_t)a.nmod};
  int rc = make_map_bf16(&map, a.digits, 3, dims, strides, box, false);
  if (rc) return rc;
  const size_t smem = residue_smem(npad);
  auto kern = a.trans ? residues_mma_kernel<MW, NL, true> : residues_mma_kernel<MW, NL, false>;
  static bool attr[2] = {false, false};
  if (!attr[a.trans ? 1 : 0]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)residue_smem(96));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return cuda_fail(e, "residue split smem attribute");
    attr[a.trans ? 1 : 0] = true;
  }
  int dev = 0, nsm = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return cuda_fail(e, "residue split attributes");
  // resident CTAs: shared memory (1 KB reserved per CTA), registers, tensor memory
  const int by_smem = smem_sm / (int)(smem + 1024);
  const int by_regs = ctas_by_registers(fa.numRegs, kResTile);
  const int by_tmem = (int)(512 / residue_tmem_cols(npad));
  const int per_sm = std::max(1, std::min({by_smem, by_regs, by_tmem}));
  const int64_t ktiles = a.trans ? (a.digit_ld + 31) / 32 : (a.digit_ld + 255) / 256;
  const int64_t ntiles = (a.trans ? (a.R + 7) / 8 : a.R) * ktiles;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)per_sm * nsm);
  kern<<<grid, kResTile, smem, s>>>(map, a.X, a.R, a.K, a.ld, a.plane_stride, a.S, S, a.nmod,
                                    npad, a.digit_ld, a.exps, status_ptr(), a.redo, a.gate);
  return cuda_fail(cudaGetLastError(), "residue split launch");
}

template <int MW>
int launch_residues_nl(const SplitArgs &a, cudaStream_t s) {
  const int bits = a.S + 3;    // |T| < m 2^(L-2) < 2^(L+1), one sign bit
  if (bits <= 128) return launch_residues_t<MW, 2>(a, s);
  if (bits <= 256) return launch_residues_t<MW, 4>(a, s);
  if (bits <= 384) return launch_residues_t<MW, 6>(a, s);
  return fail(MW_EUNSUPPORTED, "residue form: %d fixed-point bits (at most 381)", a.S);
}

// ---- reconstruction on the tensor cores ----------------------------------------------
// The product kernel leaves r_t, the balanced residue of the exact sum mod p_t,
// for every output and modulus (bfloat16).  With Q'_t = inv_t (P / p_t),
// inv_t = (P / p_t)^(-1) mod p_t, the integer X' = sum_t r_t Q'_t is congruent to
// X mod P, so X = X' - k P with k = round(X' / P) (|X| < P/8).  X' is exact:
// Q'_t = sum_n b_tn 2^(8n) in balanced bytes (P < 2^(32 top - 2): no carry out of
// byte 4 top - 1), so X' = sum_n z_n 2^(8n) with z_n = sum_t r_t b_tn, one MMA
// per tile of 128 outputs (A: 128 x D residues, B: D x 4 NL bytes), |z_n| <= 96
// 2^15 < 2^22.  The accumulators start at 1.5 2^23 (written into tensor memory
// before each product), so every partial sum is an integer in [2^23, 2^24) (exact)
// and the accumulator's bits are 0x4B400000 + z_n.  Horner joins them into
// 32-bit limbs, k comes from the limbs top-2..top of X' (|X'| < D 2^8 P), and
// X = X' + |k| (P or 2^(32 NL) - P) mod 2^(32 NL) is rounded greedily into m words.
struct CrtFuse {
  int D, top;                                      // moduli; limbs of X' below its sign
  float c64, c32;                                  // 2^(32(top - 1)) / P, 2^(32(top - 2)) / P
  int8_t qb[kCrtMaxModuli][4 * kCrtMaxLimbs];      // balanced bytes of Q'_t
  uint32_t P[kCrtMaxLimbs], nP[kCrtMaxLimbs];      // P and 2^(32 NL) - P
};

template <int NL>
struct FuseShape {
  static constexpr int NB = 4 * NL;                // byte positions: N of the MMA
  static constexpr uint32_t TCOLS = 2 * NB <= 128 ? 128u : 256u;   // two accumulators
};

// Bytes of shared memory the reconstruction kernel uses for D moduli and NL limbs
// (with the rounding's limb columns in shared memory unless LCOL).
inline size_t fuse_smem(int D, int NL, bool lcol) {
  const int D8 = (D + 7) & ~7, KM = (D8 + 15) & ~15, kc = (KM + 63) / 64;
  return 1024 + (size_t)256 * D8 + (size_t)kc * 16384 + (size_t)kc * 4 * NL * 128 +
         (lcol ? 0 : (size_t)(NL + 1) * 512) + 32;
}

template <int MW, int NL, bool LCOL>
__global__ void __launch_bounds__(128, 2)
    crt_fuse_kernel(const __grid_constant__ CUtensorMap map, const int32_t *eA, const int32_t *eB,
                    int64_t M, int64_t N, int ex0, double *C, int64_t ldc, int64_t psc,
                    unsigned int *status, const __grid_constant__ CrtFuse F) {
  constexpr int NB = FuseShape<NL>::NB;
  constexpr uint32_t TCOLS = FuseShape<NL>::TCOLS;
  const int D = F.D, D8 = (D + 7) & ~7;
  const int KM = (D8 + 15) & ~15, kc = (KM + 63) / 64;
  extern __shared__ uint8_t smem_raw[];
  // residues of a tile (128 outputs of one row) as TMA leaves them (two halves of
  // 64, D8 rows of 128 B, swizzled), the MMA's A (128 rows, K-major) and B (NB
  // rows), then (unless LCOL: each thread's local memory, when shared memory would
  // hold fewer CTAs than the tensor memory) the limbs the rounding reads by index
  uint8_t *stage = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = stage + 256 * D8;
  uint8_t *sB = sA + kc * 16384;
  uint32_t *colsm = (uint32_t *)(sB + kc * NB * 128);        // [NL + 1][128] unless LCOL
  uint64_t *bar = (uint64_t *)(colsm + (LCOL ? 0 : (NL + 1) * 128));   // residues, accumulators
  uint32_t *holder = (uint32_t *)(bar + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int idx = tid; idx < kc * 64 * NB; idx += 128) {
    const int t = idx / NB, n = idx - t * NB;
    const uint16_t v = t < D ? small_int_bf16(F.qb[t][n]) : (uint16_t)0;
    *reinterpret_cast<uint16_t *>(sB + (t >> 6) * (NB * 128) + sw128_offset(n, t & 63)) = v;
  }
  for (int t = D8; t < kc * 64; ++t)               // row tid of A past the residues
    *reinterpret_cast<uint16_t *>(sA + (t >> 6) * 16384 + sw128_offset(tid, t & 63)) = 0;
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) mbar_init(&bar[b], 1);
    fence_barrier_init();
    prefetch_map(&map);
  }
  if (warp == 0) tmem_alloc(holder, TCOLS);
  fence_proxy_async_smem();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *holder;
  // the bias 1.5 2^23 into this warp's lanes of both accumulators
  auto bias_fill = [&](int s) {
    const uint32_t ta = tmem + s * NB + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int h = 0; h < (NB + 31) / 32; ++h) {
      if (32 * h + 32 <= NB) tc_fill32(ta + 32 * h, 0x4B400000u);
      else tc_fill16(ta + 32 * h, 0x4B400000u);
    }
  };
  bias_fill(0);
  bias_fill(1);
  tc_wait_st();
  tc_fence_before();
  __syncthreads();
  const uint32_t idesc = idesc_bf16(128, NB);
  const int64_t jtiles = (N + 127) / 128, ntiles = jtiles * M;   // a tile: 128 j of one row i
  const uint32_t stage_bytes = 256u * D8;
  volatile int abort_flag = 0;

  auto issue = [&](int64_t tile) {                // one thread: the tile's residues
    const int64_t i = tile / jtiles, j0 = (tile - i * jtiles) * 128;
    mbar_arrive_expect_tx(&bar[0], stage_bytes);
    tma_load_3d(smem_u32(stage), &map, (int)j0, (int)i, 0, smem_u32(&bar[0]));
    tma_load_3d(smem_u32(stage + 128 * D8), &map, (int)j0 + 64, (int)i, 0, smem_u32(&bar[0]));
  };
  // staged residues (rows t, outputs along the row) into A (rows = outputs):
  // warp w moves outputs 32w..32w+31, eight moduli per step
  auto transpose = [&]() {
    const int c = 4 * warp + (lane >> 3), rho = lane & 7;
    const uint32_t src = smem_u32(stage) + (c >> 3) * (128 * D8) + rho * 128 + (((c & 7) ^ rho) << 4);
    const uint32_t dst = smem_u32(sA) + (8 * c + rho) * 128;
    for (int tau = 0; tau < D8 / 8; ++tau) {
      uint32_t r[4];
      ldsm_x4_trans(src + tau * 1024, r);
      stsm_x4(dst + (tau >> 3) * 16384 + (((tau & 7) ^ rho) << 4), r);
    }
  };
  uint32_t fph = 0, mph[2] = {0u, 0u};
  // X' from the accumulator of `tile`, k, X, greedy words
  auto drain = [&](int64_t tile, int s) -> bool {
    if (!__syncthreads_and(mbar_wait(&bar[1 + s], mph[s], status, &abort_flag))) return false;
    mph[s] ^= 1;
    tc_fence_after();
    const uint32_t ta = tmem + s * NB + ((uint32_t)(warp * 32) << 16);
    constexpr uint64_t K0 = 0x4B400000ull * 0x01010101ull;   // the bias in a limb's four bytes
    uint32_t U[NL];
    int64_t rc = 0;
#pragma unroll
    for (int h = 0; h < (NB + 31) / 32; ++h) {
      uint32_t z[32];
      if (32 * h + 32 <= NB) tc_ld32(ta + 32 * h, z);
      else tc_ld16(ta + 32 * h, z);
      tc_wait_ld();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (32 * h + 4 * q >= NB) break;
        const int64_t acc = rc - (int64_t)K0 + (int64_t)z[4 * q] + ((int64_t)z[4 * q + 1] << 8) +
                            ((int64_t)z[4 * q + 2] << 16) + ((int64_t)z[4 * q + 3] << 24);
        U[8 * h + q] = (uint32_t)acc;
        rc = acc >> 32;
      }
    }
    bias_fill(s);                                  // for the accumulator's next product
    tc_wait_st();
    tc_fence_before();
    const int64_t i = tile / jtiles, j = (tile - i * jtiles) * 128 + tid;
    uint32_t lcol[LCOL ? NL + 1 : 1];              // read by index: local memory
    uint32_t *col = LCOL ? lcol : colsm + tid;
    constexpr int cs = LCOL ? 1 : 128;
#pragma unroll
    for (int l = 0; l < NL; ++l) col[l * cs] = U[l];
    col[NL * cs] = (uint32_t)rc;
    const int top = F.top;
    const uint64_t hi = ((uint64_t)col[top * cs] << 32) | col[(top - 1) * cs];
    const float kf = fmaf((float)(int64_t)hi, F.c64, (float)col[(top - 2) * cs] * F.c32);
    const int k = (int)(__float_as_uint(kf + 12582912.0f) - 0x4B400000u);
    const bool pos = k > 0;
    const uint32_t ak = (uint32_t)(pos ? k : -k);
    uint64_t cy = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
      const uint64_t v = (uint64_t)ak * (pos ? F.nP[l] : F.P[l]) + U[l] + cy;
      U[l] = (uint32_t)v;
      cy = v >> 32;
    }
    if (j < N) {
      double *c = C + i * ldc + j;
      round_column<MW, NL>(U, col, cs, eA[i] + eB[j] + ex0,
                           [&](int wd, double v) { c[wd * psc] = v; });
    }
    return true;
  };

  // the next tile's residues load while this tile is moved and the previous
  // tile drains; its product runs during that drain
  int64_t cur = blockIdx.x, prev = -1;
  int slot = 0;
  bool ok = true, tma_out = false;
  uint32_t mma_out = 0;                            // accumulators with a product in flight
  if (tid == 0 && cur < ntiles) {
    issue(cur);
    tma_out = true;
  }
  while (ok && (cur < ntiles || prev >= 0)) {
    const bool have = cur < ntiles;
    if (have) {
      ok = __syncthreads_and(mbar_wait(&bar[0], fph, status, &abort_flag));
      if (!ok) break;
      fph ^= 1;
      tma_out = false;
      // the previous product has read A before A is rewritten
      if (prev >= 0 && !__syncthreads_and(mbar_wait(&bar[1 + (slot ^ 1)], mph[slot ^ 1], status,
                                                    &abort_flag))) {
        ok = false;
        break;
      }
      transpose();
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        if (cur + gridDim.x < ntiles) {
          issue(cur + gridDim.x);
          tma_out = true;
        }
        tc_fence_after();
        const uint32_t d = tmem + slot * NB;
        for (int cc = 0; cc < kc; ++cc) {
          const uint64_t ad = sw128_desc(smem_u32(sA + cc * 16384));
          const uint64_t bd = sw128_desc(smem_u32(sB + cc * NB * 128));
          for (int kk = 0; kk < 4 && 64 * cc + 16 * kk < KM; ++kk)
            tc_mma(d, ad + 2 * kk, bd + 2 * kk, idesc, 1u);   // onto the bias
        }
        tc_commit(&bar[1 + slot]);
      }
      mma_out |= 1u << slot;
    }
    if (prev >= 0) {
      ok = drain(prev, slot ^ 1);
      if (!ok) break;
      mma_out &= ~(1u << (slot ^ 1));
    }
    prev = have ? cur : -1;
    if (have) cur += gridDim.x;
    slot ^= 1;
  }
  // after a wait that gave up: let the copies and products in flight finish
  // (bounded) before the tensor memory is released
  if (!ok && tid == 0) {
    volatile int never = 0;
    if (tma_out) mbar_wait(&bar[0], fph, status, &never);
    for (int s = 0; s < 2; ++s)
      if (mma_out & (1u << s)) mbar_wait(&bar[1 + s], mph[s], status, &never);
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_free(tmem, TCOLS);
  }
}

template <int MW, int NL, bool LCOL>
int launch_crt_fuse_v(const OzakiArgs &a, const CrtFuse &F, const CUtensorMap &map, int per_sm,
                      cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(crt_fuse_kernel<MW, NL, LCOL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)fuse_smem(kCrtMaxModuli, NL, LCOL));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(crt_fuse_kernel<MW, NL, LCOL>,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return cuda_fail(e, "reconstruction smem attribute");
    attr = true;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (a.N + 127) / 128 * a.M;
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)per_sm * nsm);
  crt_fuse_kernel<MW, NL, LCOL><<<grid, 128, fuse_smem(F.D, NL, LCOL), s>>>(
      map, a.eA, a.eB, a.M, a.N, 4 - a.S_A - a.S_B, a.C, a.ldc, a.psc, status_ptr(), F);
  return cuda_fail(cudaGetLastError(), "residue reconstruction launch");
}

template <int MW, int NL>
int launch_crt_fuse_t(const OzakiArgs &a, const CrtFuse &F, const CUtensorMap &map,
                      cudaStream_t s) {
  int dev = 0, smem_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, crt_fuse_kernel<MW, NL, false>);
  if (e != cudaSuccess) return cuda_fail(e, "reconstruction attributes");
  // resident CTAs: what shared memory (1 KB reserved per CTA), registers and the
  // tensor memory (512 columns) hold; the limb columns leave shared memory only
  // when that lets more CTAs reside
  const int by_regs = ctas_by_registers(fa.numRegs, 128);
  const int by_tmem = (int)(512 / FuseShape<NL>::TCOLS);
  const int cap = std::min(by_regs, by_tmem);
  const int in_smem = smem_sm / (int)(fuse_smem(F.D, NL, false) + 1024);
  const int in_local = smem_sm / (int)(fuse_smem(F.D, NL, true) + 1024);
  if (std::min(in_local, cap) > std::min(in_smem, cap))
    return launch_crt_fuse_v<MW, NL, true>(a, F, map, std::max(1, std::min(in_local, cap)), s);
  return launch_crt_fuse_v<MW, NL, false>(a, F, map, std::max(1, std::min(in_smem, cap)), s);
}

template <int MW>
int launch_crt_fuse_m(const OzakiArgs &a, const CrtFuse &F, int NL, const CUtensorMap &map,
                      cudaStream_t s) {
  switch (NL) {
    case 8: return launch_crt_fuse_t<MW, 8>(a, F, map, s);
    case 12: return launch_crt_fuse_t<MW, 12>(a, F, map, s);
    case 16: return launch_crt_fuse_t<MW, 16>(a, F, map, s);
    case 20: return launch_crt_fuse_t<MW, 20>(a, F, map, s);
    case 24: return launch_crt_fuse_t<MW, 24>(a, F, map, s);
  }
  return fail(MW_EUNSUPPORTED, "residue form: %d limbs", NL);
}

// ---- host arithmetic on the constants ------------------------------------------
using Big = std::vector<uint32_t>;   // little-endian 32-bit limbs

void big_mul_small(Big &x, uint32_t a) {
  uint64_t c = 0;
  for (uint32_t &v : x) {
    const uint64_t s = (uint64_t)v * a + c;
    v = (uint32_t)s;
    c = s >> 32;
  }
  if (c) x.push_back((uint32_t)c);
}
uint32_t big_div_small(const Big &x, uint32_t a, Big *q) {   // returns x mod a
  uint64_t r = 0;
  if (q) q->assign(x.size(), 0);
  for (size_t i = x.size(); i-- > 0;) {
    const uint64_t cur = (r << 32) | x[i];
    if (q) (*q)[i] = (uint32_t)(cur / a);
    r = cur % a;
  }
  return (uint32_t)r;
}
uint32_t inverse_mod(uint32_t a, uint32_t p) {   // a^(-1) mod p, gcd(a, p) = 1
  int64_t t = 0, nt = 1, r = p, nr = a % p;
  while (nr) {
    const int64_t q = r / nr;
    int64_t tmp = t - q * nt; t = nt; nt = tmp;
    tmp = r - q * nr; r = nr; nr = tmp;
  }
  return (uint32_t)(t < 0 ? t + p : t);
}

}  // namespace

int crt_table_size() { return kNumModuli; }
int crt_modulus(int i) { return (i >= 0 && i < kNumModuli) ? kModuli[i] : 0; }
int crt_chunk(int i) {
  const int64_t h = crt_modulus(i) / 2;
  for (int c = 4096; c > 256; c /= 2)
    if (c * h * h <= (1 << 24)) return c;
  return 256;
}
double crt_bits(int n) {
  double b = 0;
  for (int i = 0; i < n && i < kNumModuli; ++i) b += std::log2((double)kModuli[i]);
  return b;
}

int launch_residues(const SplitArgs &a, cudaStream_t s) {
  if (a.nmod < 1 || a.nmod > kNumModuli)
    return fail(MW_EINVAL, "residue form: %d moduli (1..%d)", a.nmod, kNumModuli);
  switch (a.m) {
    case 2: return launch_residues_nl<2>(a, s);
    case 4: return launch_residues_nl<4>(a, s);
  }
  return fail(MW_EUNSUPPORTED, "residue form: m = %d (2 or 4)", a.m);
}

int launch_crt_combine(const OzakiArgs &a, cudaStream_t s) {
  const int D = a.D;
  if (D < 1 || D > kNumModuli) return fail(MW_EINVAL, "residue form: %d moduli", D);
  Big P{1};
  for (int t = 0; t < D; ++t) big_mul_small(P, kModuli[t]);
  int hb = 31;                                       // bit length of P: bl
  while (!(P.back() >> hb)) --hb;
  const int bl = 32 * (int)(P.size() - 1) + hb + 1;
  // X' = sum_t r_t Q'_t with Q'_t < P < 2^(32 top - 2); limbs of X' up to `top`
  const int top = std::max(2, (bl + 2 + 31) / 32);
  const int NL = std::max(8, (top + 3) / 4 * 4);   // limbs computed (N of the MMA / 4)
  if (NL > kCrtMaxLimbs) return fail(MW_EUNSUPPORTED, "residue form: modulus product of %d bits", bl);
  CrtFuse F{};
  F.D = D;
  F.top = top;
  for (int t = 0; t < D; ++t) {
    const uint32_t p = kModuli[t];
    Big Q;
    big_div_small(P, p, &Q);                         // P / p_t
    const uint32_t inv = inverse_mod(big_div_small(Q, p, nullptr), p);
    big_mul_small(Q, inv);                           // Q'_t = inv_t P / p_t < P
    int carry = 0;                                   // balanced bytes, least significant first
    for (int n = 0; n < 4 * NL; ++n) {
      const int byte = (size_t)(n / 4) < Q.size() ? (int)((Q[n / 4] >> (8 * (n % 4))) & 0xFF) : 0;
      const int x = byte + carry;
      carry = x >= 128;
      F.qb[t][n] = (int8_t)(x - 256 * carry);
      if (n >= 4 * top && F.qb[t][n]) return fail(MW_EUNSUPPORTED, "residue form: Q' past its limbs");
    }
    if (carry) return fail(MW_EUNSUPPORTED, "residue form: Q' past its limbs");
  }
  uint64_t borrow = 0;                               // nP = 2^(32 NL) - P
  for (int l = 0; l < NL; ++l) {
    const uint32_t pl = (size_t)l < P.size() ? P[l] : 0u;
    F.P[l] = pl;
    const uint64_t d = (uint64_t)0 - pl - borrow;
    F.nP[l] = (uint32_t)d;
    borrow = (pl | borrow) ? 1 : 0;
  }
  // P ~ Pd 2^e from its top limbs
  double Pd = 0;
  const int lo = std::max(0, (int)P.size() - 3);
  for (int l = (int)P.size() - 1; l >= lo; --l) Pd = Pd * 4294967296.0 + (double)P[l];
  const int e = 32 * lo;
  F.c64 = (float)std::ldexp(1.0 / Pd, 32 * (top - 1) - e);
  F.c32 = (float)std::ldexp(1.0 / Pd, 32 * (top - 2) - e);
  // residues: bf16 planes [t][i][j], rows of crt_ld(N); boxes of 64 outputs of
  // one row x every modulus (moduli past D, outputs past N: zeros)
  alignas(64) CUtensorMap map;
  const int64_t ld = crt_ld(a.N);
  const uint64_t dims[3] = {(uint64_t)a.N, (uint64_t)a.M, (uint64_t)D};
  const uint64_t strides[2] = {(uint64_t)ld * 2, (uint64_t)a.M * ld * 2};
  const uint32_t box[3] = {64, 1, (uint32_t)((D + 7) & ~7)};
  int rc = make_map_bf16(&map, a.partials, 3, dims, strides, box);
  if (rc) return rc;
  switch (a.m) {
    case 2: return launch_crt_fuse_m<2>(a, F, NL, map, s);
    case 4: return launch_crt_fuse_m<4>(a, F, NL, map, s);
  }
  return fail(MW_EUNSUPPORTED, "residue form: m = %d (2 or 4)", a.m);
}

}  // namespace mw
