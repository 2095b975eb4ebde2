// Steps 1-2 of the error-free summation (Section 2): a shared exponent per row
// of the logical operand, then every entry cut into S balanced pieces of w bits.
//
// Logical operand: R rows (output dimension) x K columns (reduction).  trans = 0
// reads X[r*ld + k] (k contiguous), trans = 1 reads X[k*ld + r] (r contiguous)
// and transposes through shared memory so that the pieces are written with k
// contiguous either way.
//
// Pass 1 (exponents): E'_r = max over nonzero words of ilogb+1, e'_r = min over
//   nonzero entries of the entry exponent, kept biased in int32 so that zero
//   means "nothing seen" and a memset initialises them.
// Finalize: E_r (0 for an all-zero row), spread_r = E_r - e_r, warning check.
// Pass 2 (pieces): T = sum_j trunc(x_j 2^(wS-2-E_r)) in NL 64-bit limbs (two's
//   complement), then the balanced base-2^w digits from the least significant
//   end with a carry, written as bfloat16 or double.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "mw_device.cuh"
#include "mw_pieces.cuh"

namespace mw {
namespace {

constexpr int kBias = 1 << 20;  // E and -e stored as value + kBias (> 0 for any double)

__device__ __forceinline__ void entry_exps(const double *x, int64_t plane_stride, int m,
                                           int &e_entry, bool &nonfinite) {
  e_entry = kExpZero;
  for (int j = 0; j < m; ++j) {
    const int e = exp_plus1(x[j * plane_stride]);
    if (e == kExpNonFinite) nonfinite = true;
    else if (e > e_entry) e_entry = e;
  }
}

// ---- pass 1 ------------------------------------------------------------------
// m words per entry (m = 1: the leading words only).  Kernels given a gate return
// at once while *gate == 0; their blocks loop over the work, so that a launch
// that turns out not to be needed costs few blocks.
// trans = 0: block = 256 threads along 1024 k of one row; work unit (r, k chunk).
constexpr int kRowChunk = 1024;
// operands of at least this many entries take their exponents from the leading
// words first (below it the extra launches cost more than the words saved)
constexpr int64_t kLeadMinEntries = 1 << 22;
__global__ void exps_rows_kernel(const double *__restrict__ X, int m, int64_t R, int64_t K,
                                 int64_t ld, int64_t ps, int *Eb, int *eminb,
                                 unsigned int *status, const int32_t *gate) {
  if (gate && *gate == 0) return;
  const int64_t nkc = (K + kRowChunk - 1) / kRowChunk;
  bool bad = false;
  for (int64_t u = blockIdx.x; u < R * nkc; u += gridDim.x) {
    const int64_t r = u / nkc, kc = u - r * nkc;
    int emax = kExpZero, emin = -kExpZero;
    for (int64_t k = kc * kRowChunk + threadIdx.x; k < K && k < (kc + 1) * kRowChunk;
         k += blockDim.x) {
      int e;
      entry_exps(X + r * ld + k, ps, m, e, bad);
      if (e != kExpZero) {
        emax = max(emax, e);
        emin = min(emin, e);
      }
    }
    for (int o = 16; o; o >>= 1) {
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
    }
    if ((threadIdx.x & 31) == 0 && emax != kExpZero) {
      atomicMax(Eb + r, emax + kBias);
      atomicMax(eminb + r, kBias - emin);
    }
  }
  if (bad) raise_status(status, MW_ENONFINITE);
}

// trans = 1: block = 32 (r) x 8 (k) threads; work unit: 32 columns x
// kRowsPerBlock rows of the stored K x R matrix.
constexpr int kRowsPerBlock = 32;
__global__ void exps_cols_kernel(const double *__restrict__ X, int m, int64_t R, int64_t K,
                                 int64_t ld, int64_t ps, int *Eb, int *eminb,
                                 unsigned int *status, const int32_t *gate) {
  if (gate && *gate == 0) return;
  __shared__ int smax[8][32], smin[8][32];
  const int64_t nrb = (R + 31) / 32, nkb = (K + kRowsPerBlock - 1) / kRowsPerBlock;
  bool bad = false;
  for (int64_t u = blockIdx.x; u < nrb * nkb; u += gridDim.x) {
    const int64_t kb = u / nrb, rb = u - kb * nrb;  // neighbouring blocks: neighbouring r
    const int64_t r = rb * 32 + threadIdx.x;
    const int64_t k0 = kb * kRowsPerBlock;
    int emax = kExpZero, emin = -kExpZero;
    if (r < R) {
      for (int64_t k = k0 + threadIdx.y; k < K && k < k0 + kRowsPerBlock; k += 8) {
        int e;
        entry_exps(X + k * ld + r, ps, m, e, bad);
        if (e != kExpZero) {
          emax = max(emax, e);
          emin = min(emin, e);
        }
      }
    }
    smax[threadIdx.y][threadIdx.x] = emax;
    smin[threadIdx.y][threadIdx.x] = emin;
    __syncthreads();
    if (threadIdx.y == 0 && r < R) {
      for (int i = 1; i < 8; ++i) {
        emax = max(emax, smax[i][threadIdx.x]);
        emin = min(emin, smin[i][threadIdx.x]);
      }
      if (emax != kExpZero) {
        atomicMax(Eb + r, emax + kBias);
        atomicMax(eminb + r, kBias - emin);
      }
    }
    __syncthreads();
  }
  if (bad) raise_status(status, MW_ENONFINITE);
}

// E_r and the spread from the biased maxima, then the largest spread and the
// warning (MW_WRANGE).  mode 1: the conversion only (exponents from the leading
// words, checked later); mode 2, after that check: when the operand was not
// passed over again (*redo == 0) the largest spread and the warning from the
// values already converted.
__global__ void exps_finalize_kernel(int64_t R, int *E, int *spread, int *max_spread, int range,
                                     unsigned int *status, const int32_t *redo, int mode) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= R) return;
  int Er = E[r], sp = spread[r];
  if (mode != 2 || *redo) {
    const int eb = Er, mb = sp;
    Er = eb > 0 ? eb - kBias : 0;
    sp = eb > 0 ? Er - (kBias - mb) : 0;
    E[r] = Er;
    spread[r] = sp;
  }
  if (mode == 1) return;
  if (max_spread) atomicMax(max_spread, sp);
  if (range >= 0 && sp > range) raise_status(status, MW_WRANGE);
}

// ---- pass 2 ------------------------------------------------------------------
// trans = 0: one thread per (row, pair of columns), pairs cover the padded width.
template <int MW, int NL, typename Out>
__global__ void pieces_rows_kernel(const double *__restrict__ X, int64_t R, int64_t K,
                                   int64_t ld, int64_t ps, int w, int S, Out *digits,
                                   int64_t dld, const int *E, unsigned int *status) {
  const int64_t npair = dld / 2;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= R * npair) return;
  const int64_t r = idx / npair, k = 2 * (idx % npair);
  double a[MW], b[MW];
  const bool v0 = k < K, v1 = k + 1 < K;
  const double *row = X + r * ld;
  const bool vec = v1 && ((((uintptr_t)(row + k)) & 15) == 0) && ((ps & 1) == 0);
#pragma unroll
  for (int j = 0; j < MW; ++j) {
    if (vec) {
      const double2 v = *reinterpret_cast<const double2 *>(row + j * ps + k);  // 128-bit load
      a[j] = v.x;
      b[j] = v.y;
    } else {
      a[j] = v0 ? row[j * ps + k] : 0.0;
      b[j] = v1 ? row[j * ps + k + 1] : 0.0;
    }
  }
  const int F = w * S - 2 - E[r];
  if (w == 8)
    cut_pair_w8<MW, NL, Out>(a, b, F, S, digits + r * dld + k, R * dld, status);
  else
    cut_pair<MW, NL, Out>(a, b, F, w, S, digits + r * dld + k, R * dld, status);
}

// trans = 1: 32 x 32 tiles (32 rows r, 32 columns k of the logical operand)
// staged through shared memory as doubles (m planes), then cut like trans = 0.
template <int MW, int NL, typename Out>
__global__ void pieces_cols_kernel(const double *__restrict__ X, int64_t R, int64_t K,
                                   int64_t ld, int64_t ps, int w, int S, Out *digits,
                                   int64_t dld, const int *E, unsigned int *status) {
  extern __shared__ double tile[];  // [m][32 k][33]
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int64_t r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
#pragma unroll
  for (int j = 0; j < MW; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int kl = ty + 8 * i;
      const int64_t k = k0 + kl, r = r0 + tx;
      tile[(j * 32 + kl) * 33 + tx] = (k < K && r < R) ? X[j * ps + k * ld + r] : 0.0;
    }
  __syncthreads();
  const int tid = ty * 32 + tx;
  for (int it = 0; it < 2; ++it) {
    const int e = tid + 256 * it;      // 512 pairs per tile
    const int rl = e >> 4, kl = 2 * (e & 15);
    const int64_t r = r0 + rl, k = k0 + kl;
    if (r >= R || k >= dld) continue;
    double a[MW], b[MW];
#pragma unroll
    for (int j = 0; j < MW; ++j) {
      a[j] = tile[(j * 32 + kl) * 33 + rl];
      b[j] = tile[(j * 32 + kl + 1) * 33 + rl];
    }
    const int F = w * S - 2 - E[r];
    if (w == 8)
      cut_pair_w8<MW, NL, Out>(a, b, F, S, digits + r * dld + k, R * dld, status);
    else
      cut_pair<MW, NL, Out>(a, b, F, w, S, digits + r * dld + k, R * dld, status);
  }
}

template <int MW, typename Out, int NL>
int launch_pieces(const SplitArgs &a, cudaStream_t s) {
  Out *dig = static_cast<Out *>(a.digits);
  if (!a.trans) {
    const int64_t n = a.R * (a.digit_ld / 2);
    const int threads = 256;
    pieces_rows_kernel<MW, NL, Out><<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        a.X, a.R, a.K, a.ld, a.plane_stride, a.w, a.S, dig, a.digit_ld, a.exps, status_ptr());
  } else {
    dim3 grid((unsigned)((a.R + 31) / 32), (unsigned)((a.digit_ld + 31) / 32));
    const size_t sm = (size_t)MW * 32 * 33 * sizeof(double);
    static bool attr_set = false;  // once per instantiation
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(pieces_cols_kernel<MW, NL, Out>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return cuda_fail(e, "split smem attribute");
      attr_set = true;
    }
    pieces_cols_kernel<MW, NL, Out><<<grid, dim3(32, 8), sm, s>>>(
        a.X, a.R, a.K, a.ld, a.plane_stride, a.w, a.S, dig, a.digit_ld, a.exps, status_ptr());
  }
  return cuda_fail(cudaGetLastError(), "split pieces launch");
}

template <int MW, typename Out>
int launch_pieces_nl(const SplitArgs &a, cudaStream_t s) {
  const int bits = a.w * a.S + 3;  // |T| < m 2^(wS-2) < 2^(wS+1), one sign bit
  if (bits <= 128) return launch_pieces<MW, Out, 2>(a, s);
  if (bits <= 256) return launch_pieces<MW, Out, 4>(a, s);
  if (bits <= 384) return launch_pieces<MW, Out, 6>(a, s);
  if (bits <= 512) return launch_pieces<MW, Out, 8>(a, s);
  if (bits <= 640) return launch_pieces<MW, Out, 10>(a, s);
  return fail(MW_EUNSUPPORTED, "w*S = %d too large (at most 637 bits)", a.w * a.S);
}

template <typename Out>
int launch_pieces_m(const SplitArgs &a, cudaStream_t s) {
  switch (a.m) {
    case 2: return launch_pieces_nl<2, Out>(a, s);
    case 4: return launch_pieces_nl<4, Out>(a, s);
    case 8: return launch_pieces_nl<8, Out>(a, s);
    case 16:
      // hexa doubles: bfloat16 pieces (MW_OZAKI) only
      if constexpr (std::is_same<Out, __nv_bfloat16>::value) {
        const int bits = a.w * a.S + 3;
        if (bits <= 768) return launch_pieces<16, Out, 12>(a, s);
        if (bits <= 896) return launch_pieces<16, Out, 14>(a, s);
        if (bits <= 1024) return launch_pieces<16, Out, 16>(a, s);
        return fail(MW_EUNSUPPORTED, "w*S = %d too large (at most 1021 bits)", a.w * a.S);
      } else {
        return fail(MW_EUNSUPPORTED, "m = 16 is cut into bfloat16 pieces only");
      }
  }
  return fail(MW_EINVAL, "m must be 2, 4, 8 or 16");
}

}  // namespace

// Exponents of the operand from m words per entry.  gate: the pass over every
// word after the leading words' check (runs only if *gate != 0, on a small grid:
// it is rarely needed); it accumulates onto the converted values of the first
// pass, which every biased maximum exceeds.
int launch_exps(const SplitArgs &a, int m, int mode, const int32_t *gate, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = (int64_t)(gate ? 2 : 16) * std::max(nsm, 1);
  if (!a.trans) {
    const int64_t units = a.R * ((a.K + kRowChunk - 1) / kRowChunk);
    exps_rows_kernel<<<(unsigned)std::min(units, cap), 256, 0, s>>>(
        a.X, m, a.R, a.K, a.ld, a.plane_stride, a.exps, a.spread, status_ptr(), gate);
  } else {
    const int64_t units = ((a.R + 31) / 32) * ((a.K + kRowsPerBlock - 1) / kRowsPerBlock);
    exps_cols_kernel<<<(unsigned)std::min(units, cap), dim3(32, 8), 0, s>>>(
        a.X, m, a.R, a.K, a.ld, a.plane_stride, a.exps, a.spread, status_ptr(), gate);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "split exponent launch");
  exps_finalize_kernel<<<(unsigned)((a.R + 255) / 256), 256, 0, s>>>(
      a.R, a.exps, a.spread, a.max_spread, a.range, status_ptr(), a.redo, mode);
  return cuda_fail(cudaGetLastError(), "split finalize launch");
}

int launch_split(const SplitArgs &a, bool exponents_only, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.exps, 0, sizeof(int32_t) * a.R, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.spread, 0, sizeof(int32_t) * a.R, s);
  if (e != cudaSuccess) return cuda_fail(e, "split memset");
  if (a.nmod > 0 && a.redo && !exponents_only && a.R * a.K >= kLeadMinEntries) {
    // residue form, large operands: exponents from the leading words (1/m of the
    // data), checked entry by entry by the split; only if an entry failed do the
    // exponents over every word and the split run again
    if ((e = cudaMemsetAsync(a.redo, 0, sizeof(int32_t), s)) != cudaSuccess)
      return cuda_fail(e, "split memset");
    SplitArgs b = a;
    b.gate = nullptr;
    int rc = launch_exps(b, 1, 1, nullptr, s);
    if (!rc) rc = launch_residues(b, s);
    if (!rc) rc = launch_exps(b, a.m, 2, a.redo, s);
    if (rc) return rc;
    b.redo = nullptr;
    b.gate = a.redo;
    return launch_residues(b, s);
  }
  SplitArgs b = a;
  b.redo = nullptr;
  b.gate = nullptr;
  int rc = launch_exps(b, a.m, 0, nullptr, s);
  if (rc || exponents_only) return rc;
  if (a.nmod > 0) return launch_residues(b, s);
  if (a.format == MW_DIGITS_BF16) return launch_pieces_m<__nv_bfloat16>(a, s);
  return launch_pieces_m<double>(a, s);
}

}  // namespace mw
