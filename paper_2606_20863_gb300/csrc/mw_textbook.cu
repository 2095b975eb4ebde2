// MW_TEXTBOOK: the "ordinary" m-double matrix product that Table 2 compares the
// vectorized (error-free summation) one against: every term a_ik b_kj is an
// m-double multiplication followed by an m-double addition into the running sum,
// k in order, built from the error-free transformations of floating-point
// arithmetic (Section 1's multiword arithmetic):
//   two_sum (Knuth): s = fl(a + b), e = a + b - s exactly;
//   fast_two_sum (Dekker): the same for |a| >= |b|;
//   two_prod: p = fl(a b), e = a b - p exactly (one fused multiply-add; the
//     same p and e as Dekker's splitting, which needs no fma).
// m = 2: the classic double-double addition (two two_sums, two fast_two_sums)
// and multiplication (two_prod plus the cross terms).  m = 4, 8: the exact
// partial products of each magnitude level l (a_i b_j, i + j = l < m) by
// two_prod, the level-m products rounded, all of them in level order, then
// renormalised into m words by repeated bottom-up two_sum sweeps, each sweep
// keeping its top sum as the next word and its rounding errors as the next
// sweep's terms; the addition renormalises the 2m words of both operands the
// same way.  Every operation is an explicitly rounded intrinsic, so nothing is
// contracted into a multiply-add.
//
// One thread per output, 16 x 16 outputs a CTA, 16-wide k panels of A and B
// staged in shared memory (m planes each).  The FP64 pipe bounds it.
//
// The same operations serve mw_elementwise (Table 1's add, mul and div entry by
// entry).  Division is long division, the paper giving only its operation count:
// m + 1 quotient words q_i = fl(r_0 / b_0) from the leading word of the remainder
// r (r = a at first), r = r - q_i b after each of the first m (the m-double
// product of (q_i, 0, ..., 0) and b, subtracted as an m-double addition of its
// negation; for m >= 4 the sum, which cancels in its leading words, renormalised
// once more so that its leading word leads), then the quotient words
// renormalised into m.
#include <cuda_runtime.h>

#include <algorithm>

#include "mw_device.cuh"
#include "mw_internal.h"

namespace mw {
namespace {

constexpr int kTT = 16;   // outputs per CTA side, k per panel

__device__ __forceinline__ double tb_two_sum(double a, double b, double &e) {
  const double s = __dadd_rn(a, b);
  const double bv = __dsub_rn(s, a);
  const double av = __dsub_rn(s, bv);
  e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
  return s;
}
__device__ __forceinline__ double tb_fast_two_sum(double a, double b, double &e) {
  const double s = __dadd_rn(a, b);
  e = __dsub_rn(b, __dsub_rn(s, a));
  return s;
}
__device__ __forceinline__ double tb_two_prod(double a, double b, double &e) {
  const double p = __dmul_rn(a, b);
  e = __fma_rn(a, b, -p);
  return p;
}

// n terms in level order -> m words: sweep j sums x[0..n-1-j] bottom-up; its top
// sum is word j, its rounding errors the terms of sweep j + 1.
template <int M, int N>
__device__ __forceinline__ void tb_renorm(double (&x)[N], double (&r)[M]) {
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const int n = N - j;
    if (n <= 0) {
      r[j] = 0.0;
      continue;
    }
    double s = x[n - 1];
#pragma unroll
    for (int i = n - 2; i >= 0; --i) {
      double e;
      s = tb_two_sum(x[i], s, e);
      x[i + 1] = e;
    }
    r[j] = s;
#pragma unroll
    for (int i = 0; i + 1 < n; ++i) x[i] = x[i + 1];   // the next sweep's terms
  }
}

template <int M>
__device__ __forceinline__ void tb_add(const double (&a)[M], const double (&b)[M], double (&r)[M]) {
  if constexpr (M == 2) {
    double e, f;
    double s = tb_two_sum(a[0], b[0], e);
    const double t = tb_two_sum(a[1], b[1], f);
    e = __dadd_rn(e, t);
    s = tb_fast_two_sum(s, e, e);
    e = __dadd_rn(e, f);
    s = tb_fast_two_sum(s, e, e);
    r[0] = s;
    r[1] = e;
  } else {
    double t[2 * M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      t[2 * i] = a[i];
      t[2 * i + 1] = b[i];
    }
    tb_renorm<M, 2 * M>(t, r);
  }
}

template <int M>
__device__ __forceinline__ void tb_mul(const double (&a)[M], const double (&b)[M], double (&r)[M]) {
  if constexpr (M == 2) {
    double e;
    double p = tb_two_prod(a[0], b[0], e);
    e = __dadd_rn(e, __dadd_rn(__dmul_rn(a[0], b[1]), __dmul_rn(a[1], b[0])));
    p = tb_fast_two_sum(p, e, e);
    r[0] = p;
    r[1] = e;
  } else {
    // level l: the high parts of a_i b_(l-i), then the low parts of level l-1;
    // after level m-1: the rounded level-m products a_i b_(m-i), i >= 1, and the
    // low parts of level m-1
    constexpr int NT = M * M + 2 * M - 1;
    double t[NT];
    double lo_prev[M], lo_cur[M];
    int n = 0;
#pragma unroll
    for (int l = 0; l < M; ++l) {
#pragma unroll
      for (int i = 0; i <= l; ++i) t[n++] = tb_two_prod(a[i], b[l - i], lo_cur[i]);
#pragma unroll
      for (int i = 0; i < l; ++i) t[n++] = lo_prev[i];
#pragma unroll
      for (int i = 0; i <= l; ++i) lo_prev[i] = lo_cur[i];
    }
#pragma unroll
    for (int i = 1; i < M; ++i) t[n++] = __dmul_rn(a[i], b[M - i]);
#pragma unroll
    for (int i = 0; i < M; ++i) t[n++] = lo_prev[i];
    tb_renorm<M, NT>(t, r);
  }
}

template <int M>
__device__ __forceinline__ void tb_div(const double (&a)[M], const double (&b)[M], double (&r)[M]) {
  double rem[M], q[M + 1];
#pragma unroll
  for (int w = 0; w < M; ++w) rem[w] = a[w];
#pragma unroll
  for (int i = 0; i <= M; ++i) {
    q[i] = __ddiv_rn(rem[0], b[0]);
    if (i == M) break;
    double qv[M], t[M], s[M];
    qv[0] = q[i];
#pragma unroll
    for (int w = 1; w < M; ++w) qv[w] = 0.0;
    tb_mul<M>(qv, b, t);
#pragma unroll
    for (int w = 0; w < M; ++w) t[w] = -t[w];
    tb_add<M>(rem, t, s);
    if constexpr (M > 2) {
      tb_renorm<M, M>(s, rem);
    } else {
#pragma unroll
      for (int w = 0; w < M; ++w) rem[w] = s[w];
    }
  }
  tb_renorm<M, M + 1>(q, r);
}

// C = A op B entry by entry (OP 0 add, 1 mul, 2 div), n entries, m planes each;
// one thread per entry, the loads of a plane coalesced.
template <int MW, int OP>
__global__ void __launch_bounds__(256) elementwise_kernel(const double *__restrict__ A,
                                                          int64_t psa,
                                                          const double *__restrict__ B,
                                                          int64_t psb, double *C, int64_t psc,
                                                          int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double a[MW], b[MW], r[MW];
#pragma unroll
    for (int w = 0; w < MW; ++w) {
      a[w] = A[w * psa + e];
      b[w] = B[w * psb + e];
    }
    if constexpr (OP == 0) tb_add<MW>(a, b, r);
    else if constexpr (OP == 1) tb_mul<MW>(a, b, r);
    else tb_div<MW>(a, b, r);
#pragma unroll
    for (int w = 0; w < MW; ++w) C[w * psc + e] = r[w];
  }
}

template <int MW>
int launch_elementwise_m(int op, int64_t n, const double *A, int64_t psa, const double *B,
                         int64_t psb, double *C, int64_t psc, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = (n + 255) / 256;
  const unsigned grid = (unsigned)std::min<int64_t>(blocks, (int64_t)8 * std::max(nsm, 1));
  if (op == 0) elementwise_kernel<MW, 0><<<grid, 256, 0, s>>>(A, psa, B, psb, C, psc, n);
  else if (op == 1) elementwise_kernel<MW, 1><<<grid, 256, 0, s>>>(A, psa, B, psb, C, psc, n);
  else elementwise_kernel<MW, 2><<<grid, 256, 0, s>>>(A, psa, B, psb, C, psc, n);
  return cuda_fail(cudaGetLastError(), "elementwise kernel launch");
}

// C = op(A) op(B): op(A) M x K (stored K x M when transA), op(B) K x N (stored
// N x K when transB); m planes each.
template <int MW>
__global__ void __launch_bounds__(kTT * kTT) textbook_kernel(
    const double *__restrict__ A, int64_t lda, int64_t psa, int transA,
    const double *__restrict__ B, int64_t ldb, int64_t psb, int transB, double *C, int64_t ldc,
    int64_t psc, int64_t M, int64_t N, int64_t K) {
  __shared__ double sa[MW][kTT][kTT + 1];   // [word][row][k]
  __shared__ double sb[MW][kTT][kTT + 1];   // [word][k][col]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t row = (int64_t)blockIdx.y * kTT + ty, col = (int64_t)blockIdx.x * kTT + tx;
  double acc[MW];
#pragma unroll
  for (int j = 0; j < MW; ++j) acc[j] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += kTT) {
    // panel loads: thread (ty, tx) brings element (ty, k0 + tx) of op(A) and
    // (k0 + ty, tx) of op(B), zero outside
    {
      const int64_t r = (int64_t)blockIdx.y * kTT + ty, k = k0 + tx;
      const bool in = r < M && k < K;
#pragma unroll
      for (int j = 0; j < MW; ++j)
        sa[j][ty][tx] = in ? A[j * psa + (transA ? k * lda + r : r * lda + k)] : 0.0;
    }
    {
      const int64_t k = k0 + ty, c = (int64_t)blockIdx.x * kTT + tx;
      const bool in = k < K && c < N;
#pragma unroll
      for (int j = 0; j < MW; ++j)
        sb[j][ty][tx] = in ? B[j * psb + (transB ? c * ldb + k : k * ldb + c)] : 0.0;
    }
    __syncthreads();
    const int kn = (int)(K - k0 < kTT ? K - k0 : kTT);
    for (int kk = 0; kk < kn; ++kk) {
      double a[MW], b[MW], p[MW], s[MW];
#pragma unroll
      for (int j = 0; j < MW; ++j) {
        a[j] = sa[j][ty][kk];
        b[j] = sb[j][kk][tx];
      }
      tb_mul<MW>(a, b, p);
      tb_add<MW>(acc, p, s);
#pragma unroll
      for (int j = 0; j < MW; ++j) acc[j] = s[j];
    }
    __syncthreads();
  }
  if (row < M && col < N)
#pragma unroll
    for (int j = 0; j < MW; ++j) C[j * psc + row * ldc + col] = acc[j];
}

}  // namespace

int launch_textbook(int m, int transA, int transB, int64_t M, int64_t N, int64_t K,
                    const double *A, int64_t lda, int64_t psa, const double *B, int64_t ldb,
                    int64_t psb, double *C, int64_t ldc, int64_t psc, cudaStream_t s) {
  if ((M + kTT - 1) / kTT > 65535) return fail(MW_EUNSUPPORTED, "M too large for MW_TEXTBOOK");
  dim3 grid((unsigned)((N + kTT - 1) / kTT), (unsigned)((M + kTT - 1) / kTT));
  dim3 block(kTT, kTT);
  switch (m) {
    case 2:
      textbook_kernel<2><<<grid, block, 0, s>>>(A, lda, psa, transA, B, ldb, psb, transB, C, ldc,
                                                psc, M, N, K);
      break;
    case 4:
      textbook_kernel<4><<<grid, block, 0, s>>>(A, lda, psa, transA, B, ldb, psb, transB, C, ldc,
                                                psc, M, N, K);
      break;
    case 8:
      textbook_kernel<8><<<grid, block, 0, s>>>(A, lda, psa, transA, B, ldb, psb, transB, C, ldc,
                                                psc, M, N, K);
      break;
    default:
      return fail(MW_EUNSUPPORTED, "MW_TEXTBOOK takes m = 2, 4 and 8");
  }
  return cuda_fail(cudaGetLastError(), "textbook kernel launch");
}

int launch_elementwise(int op, int m, int64_t n, const double *A, int64_t psa, const double *B,
                       int64_t psb, double *C, int64_t psc, cudaStream_t s) {
  if (n == 0) return MW_OK;
  switch (m) {
    case 2: return launch_elementwise_m<2>(op, n, A, psa, B, psb, C, psc, s);
    case 4: return launch_elementwise_m<4>(op, n, A, psa, B, psb, C, psc, s);
    case 8: return launch_elementwise_m<8>(op, n, A, psa, B, psb, C, psc, s);
  }
  return fail(MW_EUNSUPPORTED, "mw_elementwise takes m = 2, 4 and 8");
}

}  // namespace mw
