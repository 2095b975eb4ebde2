// MW_PLAIN: step 3 and 4 of the error-free summation on the FP64 pipe.
//
// Section 2 computes, for double doubles cut into 13-bit quarters,
//   s_i = sum_k sum_{j=0..i} x_{k,j} y_{k,i-j}
// in double arithmetic -- exact because the pieces have zero high bits and the
// number of terms stays below a threshold -- and then adds s_0 + s_1 + ... in
// double double arithmetic.  Here the pieces are balanced integers of w bits
// held in doubles (mw_split, format MW_DIGITS_F64) and the threshold is
// (pairs on a diagonal) * K * 2^(2w-2) <= 2^53, which mw_plan_gemm enforces, so
// every diagonal sum s_t below is exact.  Each s_t, scaled by its weight
// 2^(E_i + E_j + 4 - w(t+2)), is added into an (m+1)-word accumulator with a
// two-sum cascade (postponing renormalisation, Section 4); the accumulator is
// renormalised into m nonoverlapping words once, at the end.
//
// Tiling: a block of 16 x 16 threads computes a (16 TH) x (16 TH) tile of C,
// thread (ty, tx) the outputs (ty + 16 a, tx + 16 b); pieces are staged in
// shared memory 16 columns of the reduction at a time.
#include "mw_device.cuh"

namespace mw {
namespace {

constexpr int BKP = 16;

__device__ __forceinline__ double two_sum(double a, double b, double &e) {
  const double s = __dadd_rn(a, b);
  const double bv = __dsub_rn(s, a);
  const double av = __dsub_rn(s, bv);
  e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
  return s;
}

// Add x into the (W)-word accumulator s: top-down two-sum cascade (the error of
// each word moves to the next, the last rounding error is dropped), then a
// bottom-up sweep that keeps the words ordered by magnitude.
template <int W>
__device__ __forceinline__ void accumulate(double (&s)[W], double x) {
  double e = x;
#pragma unroll
  for (int j = 0; j < W; ++j) s[j] = two_sum(s[j], e, e);
#pragma unroll
  for (int j = W - 1; j >= 1; --j) s[j - 1] = two_sum(s[j - 1], s[j], s[j]);
}

// Renormalise W terms into M nonoverlapping words: each pass sums the remaining
// terms bottom-up with two-sum, keeps the top as the next word and the exact
// rounding errors as the terms of the next pass.
template <int W, int M>
__device__ __forceinline__ void renormalize(double (&x)[W], double (&r)[M]) {
#pragma unroll
  for (int j = 0; j < M; ++j) {
    double s = x[W - 1];
#pragma unroll
    for (int i = W - 2; i >= 0; --i) {
      double e;
      s = two_sum(x[i], s, e);
      x[i + 1] = e;
    }
    r[j] = s;
#pragma unroll
    for (int i = 0; i < W - 1; ++i) x[i] = x[i + 1];
    x[W - 1] = 0.0;
  }
}

template <int MW, int TH>
__global__ void __launch_bounds__(256, 1) plain_kernel(PlainArgs a) {
  constexpr int BT = 16 * TH;
  __shared__ double As[BKP][BT + 1];
  __shared__ double Bs[BKP][BT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * BT, j0 = (int64_t)blockIdx.x * BT;

  double st[TH][TH][MW + 1];
#pragma unroll
  for (int u = 0; u < TH; ++u)
#pragma unroll
    for (int v = 0; v < TH; ++v)
#pragma unroll
      for (int j = 0; j <= MW; ++j) st[u][v][j] = 0.0;

  int ei[TH], ej[TH];
#pragma unroll
  for (int u = 0; u < TH; ++u) {
    const int64_t i = i0 + ty + 16 * u, j = j0 + tx + 16 * u;
    ei[u] = i < a.M ? a.eA[i] : 0;
    ej[u] = j < a.N ? a.eB[j] : 0;
  }

  // load mapping: thread -> (kk = t % 16, row = t / 16 + 16 r)
  const int lk = threadIdx.x & 15, lr = threadIdx.x >> 4;
  for (int t = 0; t < a.D; ++t) {
    double acc[TH][TH];
#pragma unroll
    for (int u = 0; u < TH; ++u)
#pragma unroll
      for (int v = 0; v < TH; ++v) acc[u][v] = 0.0;
    const int plo = max(0, t - a.S_B + 1), phi = min(t, a.S_A - 1);
    for (int p = plo; p <= phi; ++p) {
      const int q = t - p;
      const double *pa = a.dA + (int64_t)p * a.M * a.Kp;
      const double *pb = a.dB + (int64_t)q * a.N * a.Kp;
      for (int64_t k0 = 0; k0 < a.Kp; k0 += BKP) {
#pragma unroll
        for (int r = 0; r < TH; ++r) {
          const int row = lr + 16 * r;
          const int64_t gi = i0 + row, gj = j0 + row;
          As[lk][row] = gi < a.M ? pa[gi * a.Kp + k0 + lk] : 0.0;
          Bs[lk][row] = gj < a.N ? pb[gj * a.Kp + k0 + lk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BKP; ++kk) {
          double x[TH], y[TH];
#pragma unroll
          for (int u = 0; u < TH; ++u) {
            x[u] = As[kk][ty + 16 * u];
            y[u] = Bs[kk][tx + 16 * u];
          }
#pragma unroll
          for (int u = 0; u < TH; ++u)
#pragma unroll
            for (int v = 0; v < TH; ++v) acc[u][v] = __fma_rn(x[u], y[v], acc[u][v]);
        }
        __syncthreads();
      }
    }
    // s_t is exact; scale by its weight (a power of two) and accumulate
#pragma unroll
    for (int u = 0; u < TH; ++u)
#pragma unroll
      for (int v = 0; v < TH; ++v)
        accumulate<MW + 1>(st[u][v], scalbn(acc[u][v], ei[u] + ej[v] + 4 - a.w * (t + 2)));
  }
#pragma unroll
  for (int u = 0; u < TH; ++u)
#pragma unroll
    for (int v = 0; v < TH; ++v) {
      const int64_t i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
      double r[MW];
      renormalize<MW + 1, MW>(st[u][v], r);
      if (i < a.M && j < a.N)
#pragma unroll
        for (int w = 0; w < MW; ++w) a.C[w * a.psc + i * a.ldc + j] = r[w];
    }
}

template <int MW, int TH>
int launch(const PlainArgs &a, cudaStream_t s) {
  constexpr int BT = 16 * TH;
  dim3 grid((unsigned)((a.N + BT - 1) / BT), (unsigned)((a.M + BT - 1) / BT));
  plain_kernel<MW, TH><<<grid, 256, 0, s>>>(a);
  return cuda_fail(cudaGetLastError(), "plain kernel launch");
}

}  // namespace

int launch_plain(const PlainArgs &a, cudaStream_t s) {
  if (a.Kp % BKP) return fail(MW_EINVAL, "padded K must be a multiple of %d", BKP);
  switch (a.m) {
    case 2: return launch<2, 4>(a, s);
    case 4: return launch<4, 2>(a, s);
    case 8: return launch<8, 2>(a, s);
  }
  return fail(MW_EINVAL, "m must be 2, 4 or 8");
}

}  // namespace mw
