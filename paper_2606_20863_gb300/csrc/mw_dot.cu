// mw_dot_batched: many m-double inner products c_i = sum_k a_ik b_ik with the
// error-free summation of Section 2 (the paper's own benchmark, Table 2, is
// 1,024 inner products of length 6,144).
//
// An inner product has no operand reuse, so the products of pieces run on the
// integer units instead of the tensor cores: one CTA per inner product,
//   1. the shared exponents E_a, E_b of the two vectors (block reduction over
//      the leading words; the cut checks them against every word and cuts
//      again in the rare case of input that is not normalised);
//   2. every entry cut into S balanced digits of w = 24 bits (|d| <= 2^23) on
//      the fixed-point grid below 2^E, as for the matrix product (m >= 8:
//      through a shared-memory column of 24-bit slots, cut_column);
//   3. each thread sums d^a_p d^b_q into int64 diagonal sums s_t, t = p + q < D
//      (|d^a d^b| <= 2^46, so a thread's share of K stays far below 2^63); the
//      block adds them up in 128 bits;
//   4. one thread fuses X = sum_t s_t 2^(w (D-1-t)) exactly and rounds
//      X 2^(E_a + E_b + 4 - w (D+1)) into m words (greedy, ties to even).
// S is a template parameter (digit positions known at compile time); the
// planner picks the smallest instance that covers the error analysis.
//
// The same kernel multiplies truncated power series (mw_convolve_batched):
// coefficient i of the product of series s, c_i = sum_{k<=i} a_k b_{i-k}, is the
// inner product of a_0..a_i with b_i..b_0, so product u = (s, i) reads a forward
// from a_0 and b backward from b_i, over i + 1 terms (Section 2's s_i are these
// convolutions).
#include <cuda.h>

#include <algorithm>
#include <cmath>

#include "mw_column.cuh"
#include "mw_device.cuh"
#include "mw_fuse.cuh"
#include "mw_internal.h"
#include "mw_pieces.cuh"

namespace mw {
namespace {

constexpr int kDotW = 24;           // digit width
constexpr int kDotThreads = 256;
constexpr int kDotExtraD = 4;       // diagonals kept beyond S (D <= S + kDotExtraD)

struct DotArgs {
  const double *A, *B;
  double *C;
  int64_t lda, psa, ldb, psb, psc;
  int64_t count, K;
  int D, range_A, range_B;
  unsigned int *status;
  // power series: count series of n = K coefficients, product u = (s, i) for
  // u < count * n, output at C[s * ldc + i]
  int conv;
  int64_t ldc;
};

// bits 24k + 23 for k = 0 .. S-2 (the bias that makes the low digits bytes-like)
template <int S>
__host__ __device__ constexpr uint64_t dot_bias(int limb) {
  uint64_t v = 0;
  for (int k = 0; k + 1 < S; ++k) {
    const int bit = kDotW * k + kDotW - 1;
    if (bit / 64 == limb) v |= 1ull << (bit % 64);
  }
  return v;
}

// Balanced digits d[p] (p = 0 most significant) of the NL-limb fixed-point
// value T, w = 24: with 2^23 added to every low digit the digits are 24-bit
// fields minus 2^23; the top digit is the signed value above them.  Returns
// false when T lies outside [-2^(wS-1), 2^(wS-1)).
template <int S, int NL>
__device__ __forceinline__ bool dot_digits(uint64_t (&T)[NL], int32_t (&d)[S]) {
  constexpr int b = kDotW * S - 1, lb = b >> 6, ob = b & 63;
  static_assert(lb < NL, "limbs cover the digits");
  const int64_t v = (int64_t)T[lb] >> ob;
  bool ok = v == 0 || v == -1;
#pragma unroll
  for (int i = lb + 1; i < NL; ++i) ok &= T[i] == (uint64_t)v;
  uint64_t H[NL];
#pragma unroll
  for (int i = 0; i < NL; ++i) H[i] = dot_bias<S>(i);
  add_limbs<NL>(T, H);
#pragma unroll
  for (int k = 0; k < S; ++k) {          // k: position from the least significant digit
    const int bit = kDotW * k, li = bit >> 6, off = bit & 63;
    uint64_t win = T[li] >> off;
    if (off != 0 && li + 1 < NL) win |= T[li + 1] << (64 - off);
    if (k + 1 < S) {
      d[S - 1 - k] = (int32_t)(win & 0xFFFFFF) - (1 << 23);
    } else {
      // the top digit: everything from bit 24 (S-1) up, sign included
      const int64_t top = (li + 1 < NL || off == 0) ? (int64_t)win : ((int64_t)T[li] >> off);
      d[0] = (int32_t)top;
    }
  }
  return ok;
}

// 8-byte asynchronous copy global -> shared (completion by commit groups)
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 128-bit (hi, lo) add
__device__ __forceinline__ void add128(uint64_t &lo, int64_t &hi, uint64_t lo2, int64_t hi2) {
  const uint64_t s = lo + lo2;
  hi = hi + hi2 + (s < lo ? 1 : 0);
  lo = s;
}

// X += V 2^sh for an unsigned 64-bit V (zero-extended)
template <int NL>
__device__ __forceinline__ void add_shifted_u(uint64_t (&X)[NL], uint64_t V, int sh) {
  const int li = sh >> 6, bo = sh & 63;
  const uint64_t lo = V << bo;
  const uint64_t hi = bo ? (V >> (64 - bo)) : 0;
  uint64_t carry = 0;
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const uint64_t a = k == li ? lo : (k == li + 1 ? hi : 0);
    const uint64_t s1 = X[k] + a;
    const uint64_t c1 = s1 < a;
    const uint64_t s2 = s1 + carry;
    carry = c1 | (s2 < carry);
    X[k] = s2;
  }
}

template <int MW, int S, int NL, int NLF>
__global__ void __launch_bounds__(kDotThreads) dot_kernel(const DotArgs a) {
  constexpr int DC = S + kDotExtraD;
  __shared__ int red_i[4][kDotThreads / 32];
  __shared__ uint64_t red_lo[kDotThreads / 32][DC];
  __shared__ int64_t red_hi[kDotThreads / 32][DC];
  __shared__ int exps[2];
  // [0]: cut again with the exponents over all words; [1]: a non-finite word;
  // [2]: an entry outside the range of its digits (raised after the last cut)
  __shared__ int red_flag[3];
  __shared__ uint32_t rcol[2 * NLF];   // the fusing thread's limbs
  extern __shared__ double stage[];   // [2 buffers][2 MW words][kDotThreads], then for
                                      // m >= 8 the threads' digit columns
  // m >= 8: each word adds its fields into this thread's column of slots
  // (cut_column) instead of a carry chain over every limb
  constexpr bool kColumn = MW >= 8;
  uint32_t *dcol = reinterpret_cast<uint32_t *>(stage + 2 * 2 * MW * kDotThreads) + threadIdx.x;
  if constexpr (kColumn)
    for (int c = 0; c < S + 3; ++c) dcol[c * kDotThreads] = 0u;   // cut_column leaves it zero
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int D = a.D;
  if (tid == 0) red_flag[0] = red_flag[1] = red_flag[2] = 0;
  __syncthreads();
  const int64_t nprod = a.conv ? a.count * a.K : a.count;
  for (int64_t i = blockIdx.x; i < nprod; i += gridDim.x) {
    // product i: inner product of length Ki of a (forward) and b (step bs)
    const int64_t s_idx = a.conv ? i / a.K : i, c_idx = a.conv ? i - s_idx * a.K : 0;
    const int64_t Ki = a.conv ? c_idx + 1 : a.K;
    const int64_t bs = a.conv ? -1 : 1;
    const double *pa = a.A + s_idx * a.lda;
    const double *pb = a.B + s_idx * a.ldb + c_idx;
    // 1. shared exponents from the leading words (an m-double's largest word is
    // its first), one read of 1/m of the data
    int ea = kExpZero, eb = kExpZero;
    for (int64_t k = tid; k < Ki; k += kDotThreads) {
      const int u = exp_plus1(pa[k]), v = exp_plus1(pb[k * bs]);
      if (u != kExpNonFinite) ea = max(ea, u);
      if (v != kExpNonFinite) eb = max(eb, v);
    }
    for (int o = 16; o; o >>= 1) {
      ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, o));
      eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, o));
    }
    if (lane == 0) { red_i[0][warp] = ea; red_i[1][warp] = eb; }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < kDotThreads / 32; ++w) {
        ea = max(ea, red_i[0][w]);
        eb = max(eb, red_i[1][w]);
      }
      exps[0] = ea == kExpZero ? 0 : ea;
      exps[1] = eb == kExpZero ? 0 : eb;
    }
    __syncthreads();
    // 2.-3. digits and this thread's diagonal sums.  The cut reads every word
    // and also finds the exponents over all words (ilogb + 1 of an entry's
    // largest word, as defined); where a later word exceeds the leading words'
    // exponent (input that is not normalised) the vectors are cut again with it.
    int64_t s[DC];
    // the words of the next entry are copied into this thread's shared slots
    // while the current one is cut (each thread reads only what it copied)
    auto slot = [&](int buf, int j) { return stage + ((buf * 2 * MW + j) * kDotThreads + tid); };
    auto fetch = [&](int64_t k, int buf) {
#pragma unroll
      for (int j = 0; j < MW; ++j) {
        cp_async8(slot(buf, j), pa + j * a.psa + k);
        cp_async8(slot(buf, MW + j), pb + j * a.psb + k * bs);
      }
    };
    for (int attempt = 0; attempt < 2; ++attempt) {
      const int Ea = exps[0], Eb = exps[1];
      const int Fa = kDotW * S - 2 - Ea, Fb = kDotW * S - 2 - Eb;
      int xa_max = kExpZero, xb_max = kExpZero, na = -kExpZero, nb = -kExpZero;
      bool nonfinite = false;
#pragma unroll
      for (int t = 0; t < DC; ++t) s[t] = 0;
      int buf = 0;
      if (tid < Ki) fetch(tid, 0);
      cp_async_commit();
      for (int64_t k = tid; k < Ki; k += kDotThreads, buf ^= 1) {
        if (k + kDotThreads < Ki) fetch(k + kDotThreads, buf ^ 1);
        cp_async_commit();
        cp_async_wait<1>();
        double xa[MW], xb[MW];
        // each entry's largest word: the largest bit pattern without the sign
        // (the order of non-negative doubles), one exponent per entry
        uint64_t ma = 0, mb = 0;
#pragma unroll
        for (int j = 0; j < MW; ++j) {
          xa[j] = *slot(buf, j);
          xb[j] = *slot(buf, MW + j);
          const uint64_t ua = (uint64_t)__double_as_longlong(xa[j]) & 0x7FFFFFFFFFFFFFFFull;
          const uint64_t ub = (uint64_t)__double_as_longlong(xb[j]) & 0x7FFFFFFFFFFFFFFFull;
          ma = ua > ma ? ua : ma;
          mb = ub > mb ? ub : mb;
        }
        const int xa_e = exp_plus1(__longlong_as_double((long long)ma));
        const int xb_e = exp_plus1(__longlong_as_double((long long)mb));
        if (xa_e == kExpNonFinite || xb_e == kExpNonFinite) nonfinite = true;
        if (xa_e != kExpZero && xa_e != kExpNonFinite) { xa_max = max(xa_max, xa_e); na = min(na, xa_e); }
        if (xb_e != kExpZero && xb_e != kExpNonFinite) { xb_max = max(xb_max, xb_e); nb = min(nb, xb_e); }
        int32_t da[S], db[S];
        if constexpr (kColumn) {
          bool ok = cut_column<MW, kDotW>(xa, Fa, S, dcol, kDotThreads,
                                          [&](int k, int32_t d) { da[S - 1 - k] = d; });
          ok &= cut_column<MW, kDotW>(xb, Fb, S, dcol, kDotThreads,
                                      [&](int k, int32_t d) { db[S - 1 - k] = d; });
          if (!ok) red_flag[2] = 1;
        } else {
          bool ok = true;
          {
            uint64_t T[NL];
            fixed_point<MW, NL>(xa, Fa, T);
            ok &= dot_digits<S, NL>(T, da);
          }
          {
            uint64_t T[NL];
            fixed_point<MW, NL>(xb, Fb, T);
            ok &= dot_digits<S, NL>(T, db);
          }
          if (!ok) red_flag[2] = 1;
        }
#pragma unroll
        for (int p = 0; p < S; ++p)
#pragma unroll
          for (int q = 0; q < S; ++q)
            if (p + q < DC && p + q < D) s[p + q] += (int64_t)da[p] * (int64_t)db[q];
      }
      cp_async_wait<0>();
      // exponents over all words: the same as the leading words' for normalised
      // input; otherwise cut again (at most once: the second pass uses them)
      for (int o = 16; o; o >>= 1) {
        xa_max = max(xa_max, __shfl_xor_sync(0xffffffffu, xa_max, o));
        xb_max = max(xb_max, __shfl_xor_sync(0xffffffffu, xb_max, o));
        na = min(na, __shfl_xor_sync(0xffffffffu, na, o));
        nb = min(nb, __shfl_xor_sync(0xffffffffu, nb, o));
      }
      if (lane == 0) {
        red_i[0][warp] = xa_max; red_i[1][warp] = xb_max; red_i[2][warp] = na; red_i[3][warp] = nb;
      }
      if (nonfinite) red_flag[1] = 1;
      __syncthreads();
      if (tid == 0) {
        for (int w = 1; w < kDotThreads / 32; ++w) {
          xa_max = max(xa_max, red_i[0][w]); xb_max = max(xb_max, red_i[1][w]);
          na = min(na, red_i[2][w]); nb = min(nb, red_i[3][w]);
        }
        const int Ta = xa_max == kExpZero ? 0 : xa_max, Tb = xb_max == kExpZero ? 0 : xb_max;
        const bool again = attempt == 0 && (Ta != Ea || Tb != Eb);
        red_flag[0] = again ? 1 : 0;
        if (!again) {
          const int sa = xa_max == kExpZero ? 0 : xa_max - na;
          const int sb = xb_max == kExpZero ? 0 : xb_max - nb;
          if ((a.range_A >= 0 && sa > a.range_A) || (a.range_B >= 0 && sb > a.range_B))
            raise_status(a.status, MW_WRANGE);
          if (red_flag[1]) raise_status(a.status, MW_ENONFINITE);
          if (red_flag[2]) raise_status(a.status, MW_ERANGE);
        }
        red_flag[1] = red_flag[2] = 0;      // every thread set its flags before the barrier
        exps[0] = Ta;
        exps[1] = Tb;
      }
      __syncthreads();
      if (red_flag[0] == 0) break;          // read by every thread before tid 0 writes it again
    }
    // block sums in 128 bits
#pragma unroll
    for (int t = 0; t < DC; ++t) {
      uint64_t lo = (uint64_t)s[t];
      int64_t hi = s[t] < 0 ? -1 : 0;
      for (int o = 16; o; o >>= 1) {
        const uint64_t lo2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const int64_t hi2 = __shfl_xor_sync(0xffffffffu, hi, o);
        add128(lo, hi, lo2, hi2);
      }
      if (lane == 0) {
        red_lo[warp][t] = lo;
        red_hi[warp][t] = hi;
      }
    }
    __syncthreads();
    // 4. fusion and rounding
    if (tid == 0) {
      uint64_t X[NLF];
#pragma unroll
      for (int k = 0; k < NLF; ++k) X[k] = 0;
      for (int t = 0; t < D && t < DC; ++t) {
        uint64_t lo = red_lo[0][t];
        int64_t hi = red_hi[0][t];
        for (int w = 1; w < kDotThreads / 32; ++w) add128(lo, hi, red_lo[w][t], red_hi[w][t]);
        const int sh = kDotW * (D - 1 - t);
        add_shifted_u<NLF>(X, lo, sh);
        add_shifted<NLF>(X, hi, sh + 64);
      }
      uint32_t U[2 * NLF];
      to_limbs32<NLF>(X, U);
      double *c = a.C + (a.conv ? s_idx * a.ldc + c_idx : i);
      const int64_t psc = a.psc;
      // exps: the exponents of the last cut (the same on both cuts but for input
      // that is not normalised)
      round_column<MW, 2 * NLF>(U, rcol, 1, exps[0] + exps[1] + 4 - kDotW * (D + 1),
                                [&](int k, double v) { c[k * psc] = v; });
    }
    __syncthreads();
  }
}

// instances: S for w = 24 and exponent spreads of up to about 80 bits
template <int MW> struct DotS;
template <> struct DotS<2> { static constexpr int lo = 4, hi = 8; };
template <> struct DotS<4> { static constexpr int lo = 8, hi = 12; };
template <> struct DotS<8> { static constexpr int lo = 17, hi = 21; };
template <> struct DotS<16> { static constexpr int lo = 35, hi = 36; };

template <int MW, int S>
int launch_dot_s(const DotArgs &a, cudaStream_t st) {
  constexpr int NL = 2 * ((kDotW * S + 3 + 127) / 128);   // carry chains exist for even NL
  // |X| < 2^(128 + w (D-1)), D <= S + kDotExtraD
  constexpr int NLF = (128 + kDotW * (S + kDotExtraD - 1) + 1 + 63) / 64;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(a.conv ? a.count * a.K : a.count, (int64_t)nsm * 8);
  constexpr size_t smem = 2 * 2 * MW * kDotThreads * sizeof(double) +
                         (MW >= 8 ? (size_t)(S + 3) * kDotThreads * sizeof(uint32_t) : 0);
  static bool attr_set = false;   // once per instance
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(dot_kernel<MW, S, NL, NLF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "dot kernel smem attribute");
    attr_set = true;
  }
  dot_kernel<MW, S, NL, NLF><<<grid, kDotThreads, smem, st>>>(a);
  return cuda_fail(cudaGetLastError(), "dot kernel launch");
}

template <int MW, int S>
int launch_dot_range(const DotArgs &a, int s_req, cudaStream_t st) {
  if constexpr (S > DotS<MW>::hi) {
    return fail(MW_EUNSUPPORTED, "inner products need %d pieces, at most %d supported", s_req,
                DotS<MW>::hi);
  } else {
    if (s_req == S) return launch_dot_s<MW, S>(a, st);
    return launch_dot_range<MW, S + 1>(a, s_req, st);
  }
}

}  // namespace

int dot_pieces_range(int m, int *lo, int *hi) {
  switch (m) {
    case 2: *lo = DotS<2>::lo; *hi = DotS<2>::hi; return MW_OK;
    case 4: *lo = DotS<4>::lo; *hi = DotS<4>::hi; return MW_OK;
    case 8: *lo = DotS<8>::lo; *hi = DotS<8>::hi; return MW_OK;
    case 16: *lo = DotS<16>::lo; *hi = DotS<16>::hi; return MW_OK;
    default: return fail(MW_EINVAL, "m = %d, must be 2, 4, 8 or 16", m);
  }
}

namespace {

int check_dot_plan(const mw_plan *plan) {
  if (!plan) return fail(MW_EINVAL, "plan is NULL");
  const mw_plan &p = *plan;
  if (p.mode != MW_DOT) return fail(MW_EINVAL, "plan mode must be MW_DOT");
  if (p.m != 2 && p.m != 4 && p.m != 8 && p.m != 16)
    return fail(MW_EINVAL, "m must be 2, 4, 8 or 16");
  if (p.w != kDotW || p.S_A != p.S_B || p.S_A < 1)
    return fail(MW_EINVAL, "MW_DOT plans have w = 24 and S_A = S_B");
  if (p.D < 1 || p.D > p.S_A + kDotExtraD || p.D > 2 * p.S_A - 1)
    return fail(MW_EINVAL, "MW_DOT plans keep at most S + %d diagonals", kDotExtraD);
  return MW_OK;
}

int launch_dot(const mw_plan &p, const DotArgs &a, cudaStream_t st) {
  switch (p.m) {
    case 2: return launch_dot_range<2, DotS<2>::lo>(a, p.S_A, st);
    case 4: return launch_dot_range<4, DotS<4>::lo>(a, p.S_A, st);
    case 8: return launch_dot_range<8, DotS<8>::lo>(a, p.S_A, st);
    default: return launch_dot_range<16, DotS<16>::lo>(a, p.S_A, st);
  }
}

}  // namespace
}  // namespace mw

using namespace mw;

extern "C" {

int mw_dot_batched(const mw_plan *plan, int64_t count, int64_t K, const double *A, int64_t lda,
                   int64_t plane_stride_a, const double *B, int64_t ldb, int64_t plane_stride_b,
                   double *C, int64_t plane_stride_c, mw_stream_t stream) {
  int rc = check_dot_plan(plan);
  if (rc) return rc;
  const mw_plan &p = *plan;
  if (count < 1 || K < 1) return fail(MW_EINVAL, "count and K must be positive");
  if (!A || !B || !C) return fail(MW_EINVAL, "NULL operand");
  if (lda < K || ldb < K) return fail(MW_EINVAL, "lda and ldb must be >= K");
  if (plane_stride_a < lda * (count - 1) + K || plane_stride_b < ldb * (count - 1) + K ||
      plane_stride_c < count)
    return fail(MW_EINVAL, "plane strides overlap");
  DotArgs a{};
  a.A = A; a.B = B; a.C = C;
  a.lda = lda; a.psa = plane_stride_a; a.ldb = ldb; a.psb = plane_stride_b;
  a.psc = plane_stride_c;
  a.count = count; a.K = K; a.D = p.D; a.range_A = p.range_A; a.range_B = p.range_B;
  a.status = status_ptr();
  return launch_dot(p, a, (cudaStream_t)stream);
}

int mw_convolve_batched(const mw_plan *plan, int64_t count, int64_t n, const double *A,
                        int64_t lda, int64_t plane_stride_a, const double *B, int64_t ldb,
                        int64_t plane_stride_b, double *C, int64_t ldc, int64_t plane_stride_c,
                        mw_stream_t stream) {
  int rc = check_dot_plan(plan);
  if (rc) return rc;
  const mw_plan &p = *plan;
  if (count < 1 || n < 1) return fail(MW_EINVAL, "count and n must be positive");
  if (!A || !B || !C) return fail(MW_EINVAL, "NULL operand");
  if (lda < n || ldb < n || ldc < n) return fail(MW_EINVAL, "lda, ldb and ldc must be >= n");
  if (plane_stride_a < lda * (count - 1) + n || plane_stride_b < ldb * (count - 1) + n ||
      plane_stride_c < ldc * (count - 1) + n)
    return fail(MW_EINVAL, "plane strides overlap");
  if (count > ((int64_t)1 << 40) / n) return fail(MW_EINVAL, "count * n too large");
  // a thread's int64 diagonal sums take ceil(n / 256) products below 2^46 each
  if ((double)p.S_A * std::ceil((double)n / kDotThreads) > 65536.0)
    return fail(MW_EUNSUPPORTED, "n = %lld too long for the inner-product kernel", (long long)n);
  DotArgs a{};
  a.A = A; a.B = B; a.C = C;
  a.lda = lda; a.psa = plane_stride_a; a.ldb = ldb; a.psb = plane_stride_b;
  a.psc = plane_stride_c; a.ldc = ldc;
  a.count = count; a.K = n; a.D = p.D; a.range_A = p.range_A; a.range_B = p.range_B;
  a.status = status_ptr();
  a.conv = 1;
  return launch_dot(p, a, (cudaStream_t)stream);
}

}  // extern "C"
