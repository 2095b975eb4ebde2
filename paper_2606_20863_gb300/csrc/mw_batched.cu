// mw_gemm_batched: many independent m-double products in the Ozaki form.
//
// The paper's application (Section 1) is power series, whose coefficient
// convolutions are many small products of uneven sizes.  One call runs every
// product of a batch with four launches, none of which needs the host to know
// more than the batch's sums (mw_batch):
//   1. prologue  (1 CTA): reads the device array of problem descriptors and
//      computes, for every problem, where its pieces, exponents and partial
//      sums live and which work items are its own (exclusive scans);
//   2. split: one warp per row of an A_i or column of a B_i -- the shared
//      exponent by a warp reduction, then the balanced pieces of the row;
//   3. product: persistent CTAs walk the work items (problem, output tile,
//      diagonal group) -- the kernel of the single product with the tile's
//      coordinates looked up per item in a table of the items' problems
//      (written by a grid-wide search after the prologue);
//   4. fusion: one thread per output, exact integer fusion and greedy
//      rounding as for the single product.
// The pieces of all problems share two row-major arrays of pitch Kpitch (the
// largest K rounded up to 64), so one tensor map per operand covers the batch;
// a tile that runs past a problem's last row reads the next rows, which only
// feed output rows/columns that are never stored.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "mw_device.cuh"
#include "mw_column.cuh"
#include "mw_fuse.cuh"
#include "mw_pieces.cuh"
#include "mw_work.cuh"

namespace mw {
namespace {

constexpr int BM = 128, BK = 64;
constexpr double kL2Budget = 48.0 * (1 << 20);  // bytes of pieces in flight
// Narrow batches run 128 x 256 tiles and put up to kMaxStack B slices of a
// problem with N <= 128 side by side in one MMA (kMaxStack - 1 zero slices
// before and after its B slices); wide batches run 128 x 128 tiles, one slice.
constexpr int kMaxStack = 8;

struct Layout {
  size_t header, info, eA, spA, eB, spB, rowtab, stripetab, outtab, pieceA, pieceB, items,
      partials, total;
  int64_t Kpitch;     // row pitch of the pieces (A when packed)
  int64_t KpitchB;    // row pitch of B's pieces
  bool packed;        // K-packed pieces (narrow batches, see BInfo)
  int64_t items_max;  // bound on the work items, from the batch sums
  int64_t rowsB;      // piece rows of B (bound: every problem with the most zero slices)
  int bn, rmax;       // tile width, most B slices per MMA
  bool narrow;   // int32 diagonal sums (D planes) or int64 group sums (G planes)
  int planes;
  int sched;     // diagonals per work item
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout_of(const mw_plan &p, const mw_batch &b) {
  Layout L{};
  L.Kpitch = L.KpitchB = round_up(b.max_K, 64);
  L.narrow = narrow_partials(p.S_A, p.S_B, p.w, b.max_K);
  L.packed = L.narrow;
  L.bn = L.narrow ? 256 : 128;
  L.rmax = L.narrow ? std::min(kMaxStack, p.D) : 1;
  L.rowsB = (int64_t)(p.S_B + 2 * (L.rmax - 1)) * b.sum_N;
  if (L.packed) {
    // a row of A: S_A slices of K8 and 64 zero columns; a row of B: S_B slices,
    // (rs - 1) K8 zero columns before them and (rs - 1) K8 + 64 (rounded up to
    // K8, at most 63 more) after them
    const int64_t K8 = round_up(b.max_K, 8);
    L.Kpitch = round_up((int64_t)p.S_A * K8 + 64, 8);
    L.KpitchB = round_up((2 * (L.rmax - 1) + p.S_B) * K8 + 128, 8);
    L.rowsB = b.sum_N;
  }
  size_t off = 0;
  L.header = off; off = a256(off + sizeof(BHeader));
  L.info = off;   off = a256(off + sizeof(BInfo) * (size_t)b.count);
  L.eA = off;     off = a256(off + 4 * (size_t)b.sum_M);
  L.spA = off;    off = a256(off + 4 * (size_t)b.sum_M);
  L.eB = off;     off = a256(off + 4 * (size_t)b.sum_N);
  L.spB = off;    off = a256(off + 4 * (size_t)b.sum_N);
  // problem of every row of the A_i, every 32-column stripe of the B_i and every
  // block of 256 outputs (lookup_tables_kernel)
  L.rowtab = off;    off = a256(off + 4 * (size_t)b.sum_M);
  L.stripetab = off; off = a256(off + 4 * (size_t)(b.sum_N / 32 + b.count + 1));
  L.outtab = off;    off = a256(off + 4 * (size_t)(b.sum_MN / 256 + 2));
  L.pieceA = off;
  off = a256(off + 2 * (size_t)(L.packed ? 1 : p.S_A) * b.sum_M * L.Kpitch);
  L.pieceB = off; off = a256(off + 2 * (size_t)L.rowsB * L.KpitchB);
  L.planes = L.narrow ? p.D : n_groups(p.D, p.group);
  // Diagonals per work item of a problem with one B slice per MMA.  The items
  // of one tile are handed out one after another, so the CTAs at work share
  // ceil(D / sched) items per tile; the pieces of the tiles in flight (row panel
  // of A and column panel of B, every slice) should fit in a share of L2, or
  // every slice pair is read from HBM.  (Stacked problems take one block of rs
  // diagonals per item.)
  if (L.narrow) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const double tile_bytes = 2.0 * ((double)L.Kpitch * BM * (L.packed ? 1 : p.S_A) +
                                     (double)L.KpitchB * L.bn * (L.packed ? 1 : p.S_B));
    const int per_tile = (int)std::min<double>(p.D, std::ceil(nsm * tile_bytes / kL2Budget));
    L.sched = (p.D + std::max(per_tile, 1) - 1) / std::max(per_tile, 1);
  } else {
    L.sched = p.group;
  }
  // ceil(M/BM) ceil(N/bn) <= MN/(BM bn) + M/BM + N/bn + 1 for every problem, and
  // at most D items per tile
  L.items_max = (int64_t)p.D *
                (b.sum_MN / (BM * L.bn) + b.sum_M / BM + b.sum_N / L.bn + b.count + 3);
  L.items = off;  off = a256(off + 4 * (size_t)L.items_max);
  L.partials = off;
  off = a256(off + (L.narrow ? 4 : 8) * (size_t)L.planes * b.sum_MN);
  L.total = off;
  return L;
}

// ---- 1. prologue --------------------------------------------------------------
__device__ int64_t block_exclusive_scan(int64_t v, int64_t *sh) {
  // 1024 threads: inclusive warp scans, then a scan of the 32 warp totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t t = sh[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;  // inclusive totals of warps 0..lane
  }
  __syncthreads();
  const int64_t before = warp ? sh[warp - 1] : 0;
  const int64_t total = sh[31];
  __syncthreads();
  sh[32] = total;
  return before + x - v;
}

__global__ void __launch_bounds__(1024) prologue_kernel(const mw_problem *probs, int count,
                                                        int D, int sched, int bn, int rmax,
                                                        int planes, int S_A, int S_B,
                                                        int packed, int64_t items_max,
                                                        mw_batch want, BInfo *info, BHeader *hdr,
                                                        unsigned int *status) {
  __shared__ int64_t sh[33];
  int64_t cM = 0, cN = 0, cMN = 0, cW = 0, cS = 0, cRB = 0;
  int bad = 0;
  for (int base = 0; base < count; base += 1024) {
    const int i = base + threadIdx.x;
    int64_t M = 0, N = 0, K = 0, w = 0;
    int tm = 0, tn = 0, rs = 1, nd = 1, G = 0, K8 = 0, Z = 0;
    mw_problem p{};
    if (i < count) {
      p = probs[i];
      M = p.M; N = p.N; K = p.K;
      const bool ok = M > 0 && N > 0 && K > 0 && K <= want.max_K && p.A && p.B && p.C &&
                      p.lda >= K && p.ldb >= N && p.ldc >= N;
      if (!ok) { bad = 1; M = N = K = 0; }
      tm = (int)((M + BM - 1) / BM);
      tn = (int)((N + bn - 1) / bn);
      // B slices side by side when the problem's N fits twice or more in a tile
      // (K-packed: column blocks of N rounded up to 8)
      const int64_t Nb = packed ? (N + 7) & ~(int64_t)7 : N;
      rs = (rmax > 1 && N > 0) ? (int)max((int64_t)1, min((int64_t)rmax, (int64_t)bn / Nb)) : 1;
      K8 = (int)((K + 7) & ~(int64_t)7);
      Z = packed ? rs - 1 : 0;
      nd = rs > 1 ? rs : sched;
      G = (D + nd - 1) / nd;
      w = (int64_t)tm * tn * G;
    }
    const int64_t pM = block_exclusive_scan(M, sh) + cM; const int64_t tM = sh[32];
    const int64_t pN = block_exclusive_scan(N, sh) + cN; const int64_t tN = sh[32];
    const int64_t pMN = block_exclusive_scan(M * N, sh) + cMN; const int64_t tMN = sh[32];
    const int64_t pW = block_exclusive_scan(w, sh) + cW; const int64_t tW = sh[32];
    const int64_t pS = block_exclusive_scan((N + 31) / 32, sh) + cS; const int64_t tS = sh[32];
    const int64_t pRB = block_exclusive_scan((int64_t)(S_B + 2 * (rs - 1)) * N, sh) + cRB;
    const int64_t tRB = sh[32];
    if (i < count) {
      BInfo b{};
      b.M = M; b.N = N; b.K = K;
      b.A = p.A; b.lda = p.lda; b.psa = p.plane_stride_a;
      b.B = p.B; b.ldb = p.ldb; b.psb = p.plane_stride_b;
      b.C = p.C; b.ldc = p.ldc; b.psc = p.plane_stride_c;
      b.rowA = packed ? pM : (int64_t)S_A * pM;
      b.rowB = packed ? pN : pRB;
      b.K8 = K8; b.Z = Z;
      b.eA = pM; b.eB = pN; b.part = (int64_t)planes * pMN; b.work = pW; b.outs = pMN; b.stripes = pS;
      b.tiles_m = tm; b.tiles_n = tn; b.KB = (int)((K + BK - 1) / BK);
      b.rs = rs; b.nd = nd; b.G = G;
      info[i] = b;
    }
    cM += tM; cN += tN; cMN += tMN; cW += tW; cS += tS; cRB += tRB;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) {
    if (cM != want.sum_M || cN != want.sum_N || cMN != want.sum_MN || cW > items_max) bad = 1;
    hdr->sum_M = cM; hdr->sum_N = cN; hdr->sum_MN = cMN; hdr->total_work = bad ? 0 : cW;
    hdr->sum_stripes = cS;
    hdr->bad = bad;
    if (bad) raise_status(status, MW_EINVAL);
  }
}

// The problem of every work item (items are numbered problem by problem), so
// that the product kernel finds an item's problem with one load.
__global__ void __launch_bounds__(256) item_table_kernel(const BInfo *info, const BHeader *hdr,
                                                         int count, int32_t *table) {
  if (hdr->bad) return;
  const int64_t total = hdr->total_work;   // at most items_max (the prologue checks)
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total;
       u += (int64_t)gridDim.x * blockDim.x)
    table[u] = find_problem(info, count, u, [](const BInfo &b) { return b.work; });
}

// The problem of every row of the A_i (rows numbered problem by problem), of
// every 32-column stripe of the B_i and of every block of 256 outputs (the
// block's first output), one warp per problem: the split and fusion kernels
// read it with one load instead of a binary search over the descriptors.
__global__ void __launch_bounds__(256) lookup_tables_kernel(const BInfo *info, const BHeader *hdr,
                                                            int count, int32_t *rowtab,
                                                            int32_t *stripetab, int32_t *outtab) {
  if (hdr->bad) return;
  const int lane = threadIdx.x & 31;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const BInfo &b = info[i];
    for (int64_t r = lane; r < b.M; r += 32) rowtab[b.eA + r] = (int32_t)i;
    for (int64_t t = lane; t < (b.N + 31) / 32; t += 32) stripetab[b.stripes + t] = (int32_t)i;
    const int64_t first = (b.outs + 255) >> 8, last = (b.outs + b.M * b.N - 1) >> 8;
    for (int64_t blk = first + lane; blk <= last; blk += 32) outtab[blk] = (int32_t)i;
  }
}

// ---- 2. split ---------------------------------------------------------------------
// Rows of the A_i: one warp per row (k contiguous, coalesced reads); the shared
// exponent by a warp reduction (for m >= 8 over the leading words, checked
// against every word while cutting), then the balanced pieces of the row.  W8: the
// w = 8 digit cutter (compiled alone, so the kernel's code stays small).  Columns
// from K up to K rounded to 64 are zero; the product never reads past them.
template <int MW, int NL, bool W8>
__global__ void __launch_bounds__(256, 4) batch_split_rows_kernel(
    const BInfo *info, const BHeader *hdr, int count, int w, int S, int64_t Kpitch,
    __nv_bfloat16 *pieceA, int32_t *eA, int32_t *spA, int32_t *max_spread, int range,
    int exps_only, int packed, const int32_t *rowtab, unsigned int *status) {
  if (hdr->bad) return;
  // m >= 8, w = 8: each word adds its fields into this thread's column of slots
  // (cut_column) instead of a carry chain over every limb
  constexpr bool kColumn = W8 && MW >= 8;
  constexpr int kSlots = kColumn ? (64 * NL - 8) / 24 + 4 : 1;   // S <= 8 NL
  __shared__ uint32_t slots[kSlots][256];
  if constexpr (kColumn)
    for (int c = 0; c < kSlots; ++c) slots[c][threadIdx.x] = 0u;   // cut_column leaves it zero
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
       task < hdr->sum_M; task += nwarps) {
    const int i = rowtab[task];
    const BInfo &b = info[i];
    const int64_t r = task - b.eA, K = b.K;
    const double *base = b.A + r * b.lda;
    // 1. the shared exponent.  Column cuts (m >= 8) take it from the leading
    //    words (1/m of the data) and the cut below checks it against every
    //    word; the spread measurement and the other cutters read every word.
    const bool lead = kColumn && !exps_only;
    int emax = kExpZero, emin = -kExpZero;
    bool nonfinite = false;
    for (int64_t k = lane; k < K; k += 32) {
      int e = kExpZero;
#pragma unroll
      for (int j = 0; j < MW; ++j) {
        if (lead && j > 0) break;
        const int x = exp_plus1(base[j * b.psa + k]);
        if (x == kExpNonFinite) nonfinite = true;
        else e = max(e, x);
      }
      if (e != kExpZero) { emax = max(emax, e); emin = min(emin, e); }
    }
    for (int o = 16; o; o >>= 1) {
      emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
    }
    int E = emax == kExpZero ? 0 : emax;
    auto finish = [&](int Ef, int sp, bool nonfin) {   // exponent, spread and flags of the row
      if (nonfin) raise_status(status, MW_ENONFINITE);
      if (lane == 0) {
        eA[task] = Ef;
        spA[task] = sp;
        atomicMax(max_spread, sp);
        if (range >= 0 && sp > range) raise_status(status, MW_WRANGE);
      }
    };
    if (!lead) finish(E, emax == kExpZero ? 0 : emax - emin, nonfinite);
    if (exps_only) continue;
    // slice p of entry k at dst + p plane + k: planes of M rows, or (K-packed) the
    // row's slices back to back, K8 apart, then 64 zero columns
    __nv_bfloat16 *dst = pieceA + (b.rowA + r) * Kpitch;
    const int64_t plane = packed ? (int64_t)b.K8 : b.M * Kpitch;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    const int64_t Kp = packed ? (int64_t)b.K8 : (K + 63) & ~(int64_t)63;
    if (packed)
      for (int c = lane; c < 64; c += 32) dst[(int64_t)S * b.K8 + c] = zero;
    for (int attempt = 0; attempt < 2; ++attempt) {
      const int F = w * S - 2 - E;
      int tmax = kExpZero, tmin = -kExpZero;       // entry exponents over every word
      bool tnonfinite = false, out_of_range = false;
      for (int64_t k = lane; k < Kp; k += 32) {
        if (k >= K) {  // zero padding: no arithmetic
          if (attempt == 0) {
            __nv_bfloat16 *q = dst + k;
            for (int p = 0; p < S; ++p, q += plane) *q = zero;
          }
          continue;
        }
        double x[MW];
#pragma unroll
        for (int j = 0; j < MW; ++j) x[j] = base[j * b.psa + k];
        if constexpr (kColumn) {
          // the entry's largest word: the largest bit pattern without the sign
          uint64_t mx = 0;
#pragma unroll
          for (int j = 0; j < MW; ++j) {
            const uint64_t u = (uint64_t)__double_as_longlong(x[j]) & 0x7FFFFFFFFFFFFFFFull;
            mx = u > mx ? u : mx;
          }
          const int xe = exp_plus1(__longlong_as_double((long long)mx));
          if (xe == kExpNonFinite) tnonfinite = true;
          else if (xe != kExpZero) { tmax = max(tmax, xe); tmin = min(tmin, xe); }
          // digits from the least significant (piece S-1) up
          uint16_t *q = reinterpret_cast<uint16_t *>(dst + k) + (int64_t)(S - 1) * plane;
          if (!cut_column<MW, 8>(x, F, S, &slots[0][threadIdx.x], 256, [&](int, int32_t d) {
                *q = small_int_bf16(d);
                q -= plane;
              }))
            out_of_range = true;
        } else if constexpr (W8) {
          cut_one_w8<MW, NL, __nv_bfloat16>(x, F, S, dst + k, plane, status);
        } else {
          cut_one<MW, NL, __nv_bfloat16>(x, F, w, S, dst + k, plane, status);
        }
      }
      if constexpr (kColumn) {   // (here lead: the spread measurement never cuts)
        // the exponent over every word: the leading words' one for normalised
        // input; otherwise the row is cut again with it
        for (int o = 16; o; o >>= 1) {
          tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
          tmin = min(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
        }
        const int Et = tmax == kExpZero ? 0 : tmax;
        if (Et != E && attempt == 0) {
          E = Et;
          continue;
        }
        if (out_of_range) raise_status(status, MW_ERANGE);
        finish(Et, tmax == kExpZero ? 0 : tmax - tmin,
               __any_sync(0xffffffffu, tnonfinite || nonfinite));
      }
      break;
    }
  }
}

// Columns of the B_i: one CTA (32 x 8 threads) per 32-column stripe of one
// problem.  Pass 1 reads rows of the stripe (coalesced) and reduces the column
// exponents in shared memory (for m >= 8 from the leading words, checked
// against every word in pass 2, which cuts the stripe again if a later word is
// larger); pass 2 stages 16 x 32 tiles of the stripe in shared memory and cuts
// them so that the pieces are written k-contiguous.
template <int MW, int NL, bool W8>
__global__ void __launch_bounds__(256, 2) batch_split_cols_kernel(
    const BInfo *info, const BHeader *hdr, int count, int w, int S, int64_t Kpitch,
    __nv_bfloat16 *pieceB, int32_t *eB, int32_t *spB, int32_t *max_spread, int range,
    int exps_only, int packed, const int32_t *stripetab, unsigned int *status) {
  extern __shared__ double tile[];              // [MW][16 k][33], then for the column
                                                // cut the threads' slots
  __shared__ int smax[8][32], smin[8][32], sE[32];
  __shared__ int tmx[32], tmn[32], redo, rflag[2];   // exponents over every word, flags
  constexpr bool kColumn = W8 && MW >= 8;     // as in the row kernel
  uint32_t *slots = reinterpret_cast<uint32_t *>(tile + MW * 16 * 33) + threadIdx.x;
  if constexpr (kColumn)
    for (int c = 0; c < (64 * NL - 8) / 24 + 4; ++c) slots[c * 256] = 0u;   // left zero by cut_column
  if (hdr->bad) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t task = blockIdx.x; task < hdr->sum_stripes; task += gridDim.x) {
    const int i = stripetab[task];
    const BInfo &b = info[i];
    const int64_t j0 = (task - b.stripes) * 32, K = b.K;
    const int64_t j = j0 + tx;
    // pass 1: column cuts (m >= 8) take the exponents from the leading words and
    // check them against every word in pass 2, as in the row kernel
    const bool lead = kColumn && !exps_only;
    int emax = kExpZero, emin = -kExpZero;
    bool nonfinite = false;
    if (j < b.N)
#pragma unroll 4
      for (int64_t k = ty; k < K; k += 8) {
        int e = kExpZero;
#pragma unroll
        for (int q = 0; q < MW; ++q) {
          if (lead && q > 0) break;
          const int x = exp_plus1(b.B[q * b.psb + k * b.ldb + j]);
          if (x == kExpNonFinite) nonfinite = true;
          else e = max(e, x);
        }
        if (e != kExpZero) { emax = max(emax, e); emin = min(emin, e); }
      }
    if (nonfinite) raise_status(status, MW_ENONFINITE);
    smax[ty][tx] = emax;
    smin[ty][tx] = emin;
    __syncthreads();
    if (ty == 0) {
      for (int y = 1; y < 8; ++y) {
        emax = max(emax, smax[y][tx]);
        emin = min(emin, smin[y][tx]);
      }
      const int E = emax == kExpZero ? 0 : emax;
      const int sp = emax == kExpZero ? 0 : emax - emin;
      sE[tx] = E;
      if (j < b.N && !lead) {
        eB[b.eB + j] = E;
        spB[b.eB + j] = sp;
        atomicMax(max_spread, sp);
        if (range >= 0 && sp > range) raise_status(status, MW_WRANGE);
      }
    }
    __syncthreads();
    // K-packed: the row of column j holds zk zeros, slices S-1 .. 0, zh zeros
    const int64_t K8 = b.K8, zk = (int64_t)b.Z * K8;
    const int64_t zh = packed ? ((int64_t)(b.rs - 1) * K8 + 64 + K8 - 1) / K8 * K8 : 0;
    if (!exps_only && packed) {
      const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
      const int64_t zt = zk + zh;                  // zero columns of a row
      for (int64_t e = threadIdx.x; e < 32 * zt; e += 256) {
        const int64_t jl = e / zt, pos = e - jl * zt;
        if (j0 + jl < b.N)
          pieceB[(b.rowB + j0 + jl) * Kpitch + (pos < zk ? pos : pos + (int64_t)S * K8)] = zero;
      }
    }
    if (!exps_only) for (int attempt = 0; attempt < 2; ++attempt) {
      const int64_t plane = packed ? -K8 : b.N * Kpitch;
      const int64_t Kp = packed ? (K8 + 15) & ~(int64_t)15 : (K + 63) & ~(int64_t)63;
      if (ty == 0) {
        tmx[tx] = kExpZero;
        tmn[tx] = -kExpZero;
      }
      if (threadIdx.x == 0) redo = rflag[0] = rflag[1] = 0;
      // entry exponents over every word of this thread's two columns
      int tmax[2] = {kExpZero, kExpZero}, tmin[2] = {-kExpZero, -kExpZero};
      // this thread's share of the next tile (rows ty, ty + 8), loaded while the
      // current one is cut
      double nxt[MW][2];
      auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int q = 0; q < MW; ++q)
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int64_t k = k0 + ty + 8 * u;
            nxt[q][u] = (k < K && j < b.N) ? b.B[q * b.psb + k * b.ldb + j] : 0.0;
          }
      };
      fetch(0);
      for (int64_t k0 = 0; k0 < Kp; k0 += 16) {
#pragma unroll
        for (int q = 0; q < MW; ++q)
#pragma unroll
          for (int u = 0; u < 2; ++u) tile[(q * 16 + ty + 8 * u) * 33 + tx] = nxt[q][u];
        __syncthreads();
        if (k0 + 16 < Kp) fetch(k0 + 16);
#pragma unroll
        for (int it = 0; it < 2; ++it) {
          const int e = threadIdx.x + 256 * it;   // 512 entries per tile, k fastest
          const int jl = e >> 4, kl = e & 15;
          const int64_t jj = j0 + jl, k = k0 + kl;
          if (jj >= b.N || (packed && k >= K8)) continue;
          // slice q of column jj at row rowB + (q + rs - 1) N + jj, the rs - 1 slices
          // before slice 0 and after slice S - 1 zero; K-packed: at column
          // (Z + S - 1 - q) K8 + k of row rowB + jj
          __nv_bfloat16 *dst = packed
              ? pieceB + (b.rowB + jj) * Kpitch + (zk + (int64_t)(S - 1) * K8) + k
              : pieceB + (b.rowB + (int64_t)(b.rs - 1) * b.N + jj) * Kpitch + k;
          const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
          if (attempt == 0) {
            if (!packed)
              for (int p = 1; p < b.rs; ++p) {
                dst[-p * plane] = zero;
                dst[(S - 1 + p) * plane] = zero;
              }
            if (k >= K) {
              __nv_bfloat16 *q = dst;
              for (int p = 0; p < S; ++p, q += plane) *q = zero;
            }
          }
          if (k >= K) continue;
          double x[MW];
#pragma unroll
          for (int q = 0; q < MW; ++q) x[q] = tile[(q * 16 + kl) * 33 + jl];
          const int F = w * S - 2 - sE[jl];
          if constexpr (kColumn) {
            uint64_t mx = 0;                        // the entry's largest word
#pragma unroll
            for (int q = 0; q < MW; ++q) {
              const uint64_t u = (uint64_t)__double_as_longlong(x[q]) & 0x7FFFFFFFFFFFFFFFull;
              mx = u > mx ? u : mx;
            }
            const int xe = exp_plus1(__longlong_as_double((long long)mx));
            if (xe == kExpNonFinite) rflag[0] = 1;
            else if (xe != kExpZero) { tmax[it] = max(tmax[it], xe); tmin[it] = min(tmin[it], xe); }
            // digits from the least significant (piece S-1) up
            uint16_t *q = reinterpret_cast<uint16_t *>(dst) + (int64_t)(S - 1) * plane;
            if (!cut_column<MW, 8>(x, F, S, slots, 256, [&](int, int32_t d) {
                  *q = small_int_bf16(d);
                  q -= plane;
                }))
              rflag[1] = 1;
          } else if constexpr (W8) {
            cut_one_w8<MW, NL, __nv_bfloat16>(x, F, S, dst, plane, status);
          } else {
            cut_one<MW, NL, __nv_bfloat16>(x, F, w, S, dst, plane, status);
          }
        }
        __syncthreads();
      }
      if constexpr (kColumn) {   // (here lead: the spread measurement never cuts)
        // exponents over every word against the leading words' (normalised input:
        // equal; otherwise the stripe is cut again with them)
#pragma unroll
        for (int it = 0; it < 2; ++it) {
          const int jl = (threadIdx.x >> 4) + 16 * it;
          atomicMax(&tmx[jl], tmax[it]);
          atomicMin(&tmn[jl], tmin[it]);
        }
        __syncthreads();
        if (ty == 0) {
          const int Et = tmx[tx] == kExpZero ? 0 : tmx[tx];
          if (j < b.N && Et != sE[tx]) redo = 1;
        }
        __syncthreads();
        if (redo && attempt == 0) {
          if (ty == 0) sE[tx] = tmx[tx] == kExpZero ? 0 : tmx[tx];
          __syncthreads();
          continue;
        }
        if (ty == 0 && j < b.N) {
          const int Et = tmx[tx] == kExpZero ? 0 : tmx[tx];
          const int sp = tmx[tx] == kExpZero ? 0 : tmx[tx] - tmn[tx];
          eB[b.eB + j] = Et;
          spB[b.eB + j] = sp;
          atomicMax(max_spread, sp);
          if (range >= 0 && sp > range) raise_status(status, MW_WRANGE);
        }
        if (threadIdx.x == 0) {
          if (rflag[0]) raise_status(status, MW_ENONFINITE);
          if (rflag[1]) raise_status(status, MW_ERANGE);
        }
      }
      break;
    }
    __syncthreads();
  }
}

// ---- 4. fusion ------------------------------------------------------------------------
// One thread per output, outputs numbered problem by problem and, inside a
// problem, column by column (the order of the column-major partial planes),
// so consecutive threads read consecutive partial sums whatever the sizes.
template <int MW, int NL, bool NARROW>
__global__ void __launch_bounds__(256, 3) batch_combine_kernel(const BInfo *info, const BHeader *hdr,
                                                            int count, const void *partials,
                                                            const int32_t *eA, const int32_t *eB,
                                                            int G, int group, int D, int w,
                                                            const int32_t *outtab) {
  if (hdr->bad) return;
  __shared__ uint32_t limbs[2 * NL][256];          // this thread's column: limbs[*][threadIdx.x]
  const int64_t total = hdr->sum_MN;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = base + threadIdx.x;
    if (f >= total) continue;
    int i = outtab[base >> 8];                              // problem of the block's first output
    while (i + 1 < count && info[i + 1].outs <= f) ++i;   // at most a few steps
    const BInfo &b = info[i];
    const int64_t o = f - b.outs;                           // = j * M + r
    int64_t j, r;
    if (o <= 0xFFFFFFFFll && b.M <= 0xFFFFFFFFll) {         // 32-bit division when it fits
      j = (uint32_t)o / (uint32_t)b.M;
      r = o - j * b.M;
    } else {
      j = o / b.M;
      r = o - j * b.M;
    }
    uint32_t U[2 * NL];
    if (NARROW && w == 8) {
      fuse_w8<2 * NL>(U, static_cast<const int32_t *>(partials) + b.part + o, b.N * b.M, D);
    } else {
      uint64_t X[NL];
#pragma unroll
      for (int k = 0; k < NL; ++k) X[k] = 0;
      if constexpr (NARROW) {
        fuse_diagonals<NL>(X, static_cast<const int32_t *>(partials) + b.part + o, b.N * b.M, D,
                           group, w);
      } else {
        const int64_t *p = static_cast<const int64_t *>(partials) + b.part + o;
        for (int g = 0; g < G; ++g) {
          const int t1 = min(D, (g + 1) * group) - 1;
          add_shifted<NL>(X, p[(int64_t)g * b.N * b.M], w * (D - 1 - t1));
        }
      }
      to_limbs32<NL>(X, U);
    }
    double *c = b.C + r * b.ldc + j;
    const int64_t psc = b.psc;
    round_column<MW, 2 * NL>(U, &limbs[0][threadIdx.x], 256,
                             eA[b.eA + r] + eB[b.eB + j] + 4 - w * (D + 1),
                             [&](int k, double v) { c[k * psc] = v; });
  }
}

int grid_for(int per_sm) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm * per_sm;
}

int check_batch(const mw_plan *p, const mw_batch *b) {
  if (!p || !b) return fail(MW_EINVAL, "plan/batch is NULL");
  if (p->mode != MW_OZAKI) return fail(MW_EUNSUPPORTED, "batches run in the Ozaki form");
  if (p->m != 2 && p->m != 4 && p->m != 8 && p->m != 16)
    return fail(MW_EINVAL, "batches take m = 2, 4, 8 or 16");
  if (b->count < 1 || b->sum_M < 1 || b->sum_N < 1 || b->max_K < 1)
    return fail(MW_EINVAL, "empty batch");
  if (p->w < 2 || p->w > 8 || (int64_t)p->chunk << (2 * p->w - 2) > (1 << 24) || p->chunk % 64)
    return fail(MW_EINVAL, "bad w/chunk");
  if (p->S_A < 1 || p->S_B < 1 || p->D < 1 || p->group < 1) return fail(MW_EINVAL, "bad plan");
  const int S_min = std::min(p->S_A, p->S_B);
  const double bits = std::ceil(std::log2((double)S_min * (double)b->max_K)) + 2 * p->w - 2;
  if (bits > 62 || bits + (double)p->w * (p->group - 1) > 62)
    return fail(MW_EINVAL, "group %d too large for K = %lld", p->group, (long long)b->max_K);
  if ((int64_t)p->S_A * b->sum_M > 0x7fffffffLL ||
      (int64_t)(p->S_B + 2 * (kMaxStack - 1)) * b->sum_N > 0x7fffffffLL)
    return fail(MW_EUNSUPPORTED, "batch too large for 32-bit piece rows");
  return MW_OK;
}

template <int MW, int NL, bool W8>
int launch_split_w(const BInfo *info, const BHeader *hdr, const mw_batch &b, const mw_plan &p,
                   uint8_t *w8, const Layout &L, int exps_only, cudaStream_t s) {
  BHeader *h = reinterpret_cast<BHeader *>(w8 + L.header);
  batch_split_rows_kernel<MW, NL, W8><<<grid_for(8), 256, 0, s>>>(
      info, hdr, b.count, p.w, p.S_A, L.Kpitch, reinterpret_cast<__nv_bfloat16 *>(w8 + L.pieceA),
      reinterpret_cast<int32_t *>(w8 + L.eA), reinterpret_cast<int32_t *>(w8 + L.spA),
      h->max_spread, p.range_A, exps_only, L.packed ? 1 : 0,
      reinterpret_cast<const int32_t *>(w8 + L.rowtab), status_ptr());
  // the 16-row tile, then (w = 8, m >= 8) 256 columns of (64 NL - 8) / 24 + 4 slots
  const size_t sm = (size_t)MW * 16 * 33 * sizeof(double) +
                    (W8 && MW >= 8 ? (size_t)((64 * NL - 8) / 24 + 4) * 256 * sizeof(uint32_t) : 0);
  static bool attr_set = false;  // once per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(batch_split_cols_kernel<MW, NL, W8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_fail(e, "batched split smem attribute");
    attr_set = true;
  }
  batch_split_cols_kernel<MW, NL, W8><<<grid_for(2), 256, sm, s>>>(
      info, hdr, b.count, p.w, p.S_B, L.KpitchB, reinterpret_cast<__nv_bfloat16 *>(w8 + L.pieceB),
      reinterpret_cast<int32_t *>(w8 + L.eB), reinterpret_cast<int32_t *>(w8 + L.spB),
      h->max_spread + 1, p.range_B, exps_only, L.packed ? 1 : 0,
      reinterpret_cast<const int32_t *>(w8 + L.stripetab), status_ptr());
  return MW_OK;
}

template <int MW, int NL>
int launch_split_nl(const BInfo *info, const BHeader *hdr, const mw_batch &b, const mw_plan &p,
                    uint8_t *w8, const Layout &L, int exps_only, cudaStream_t s) {
  return p.w == 8 ? launch_split_w<MW, NL, true>(info, hdr, b, p, w8, L, exps_only, s)
                  : launch_split_w<MW, NL, false>(info, hdr, b, p, w8, L, exps_only, s);
}

int run_front(const mw_plan &p, const mw_batch &b, const mw_problem *probs, void *ws,
              const Layout &L, int exps_only, cudaStream_t s) {
  uint8_t *w8 = static_cast<uint8_t *>(ws);
  BInfo *info = reinterpret_cast<BInfo *>(w8 + L.info);
  BHeader *hdr = reinterpret_cast<BHeader *>(w8 + L.header);
  cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(BHeader), s);
  if (e != cudaSuccess) return cuda_fail(e, "batch header memset");
  prologue_kernel<<<1, 1024, 0, s>>>(probs, b.count, p.D, L.sched, L.bn, L.rmax, L.planes, p.S_A,
                                     p.S_B, L.packed ? 1 : 0, L.items_max, b, info, hdr,
                                     status_ptr());
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch prologue launch");
  lookup_tables_kernel<<<(unsigned)std::min<int64_t>((b.count + 7) / 8, grid_for(4)), 256, 0, s>>>(
      info, hdr, b.count, reinterpret_cast<int32_t *>(w8 + L.rowtab),
      reinterpret_cast<int32_t *>(w8 + L.stripetab), reinterpret_cast<int32_t *>(w8 + L.outtab));
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch lookup tables launch");
  if (!exps_only) {
    item_table_kernel<<<grid_for(4), 256, 0, s>>>(info, hdr, b.count,
                                                  reinterpret_cast<int32_t *>(w8 + L.items));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch item table launch");
  }
  const int bits = p.w * std::max(p.S_A, p.S_B) + 3;
  int nl = bits <= 128 ? 2 : bits <= 256 ? 4 : bits <= 384 ? 6 : bits <= 512 ? 8 : bits <= 640 ? 10 : 0;
  if (p.m == 16) nl = bits <= 896 ? 14 : bits <= 1024 ? 16 : 0;   // 52 x 16 bits and more
  if (!nl) return fail(MW_EUNSUPPORTED, "w*S too large");
#define MW_SPLIT_CASE(MWV, NLV) \
  if (p.m == MWV && nl == NLV) { int rc = launch_split_nl<MWV, NLV>(info, hdr, b, p, w8, L, exps_only, s); if (rc) return rc; }
  MW_SPLIT_CASE(2, 2) MW_SPLIT_CASE(2, 4) MW_SPLIT_CASE(2, 6) MW_SPLIT_CASE(2, 8) MW_SPLIT_CASE(2, 10)
  MW_SPLIT_CASE(4, 2) MW_SPLIT_CASE(4, 4) MW_SPLIT_CASE(4, 6) MW_SPLIT_CASE(4, 8) MW_SPLIT_CASE(4, 10)
  MW_SPLIT_CASE(8, 2) MW_SPLIT_CASE(8, 4) MW_SPLIT_CASE(8, 6) MW_SPLIT_CASE(8, 8) MW_SPLIT_CASE(8, 10)
  MW_SPLIT_CASE(16, 14) MW_SPLIT_CASE(16, 16)
#undef MW_SPLIT_CASE
  return cuda_fail(cudaGetLastError(), "batch split launch");
}

template <int MW, int NL>
void launch_combine_b(const BInfo *info, const BHeader *hdr, const mw_batch &b,
                      const mw_plan &p, uint8_t *w8, const Layout &L, cudaStream_t s) {
  const int32_t *eA = reinterpret_cast<const int32_t *>(w8 + L.eA);
  const int32_t *eB = reinterpret_cast<const int32_t *>(w8 + L.eB);
  if (L.narrow)
    batch_combine_kernel<MW, NL, true><<<grid_for(3), 256, 0, s>>>(
        info, hdr, b.count, w8 + L.partials, eA, eB, n_groups(p.D, p.group), p.group, p.D, p.w,
        reinterpret_cast<const int32_t *>(w8 + L.outtab));
  else
    batch_combine_kernel<MW, NL, false><<<grid_for(3), 256, 0, s>>>(
        info, hdr, b.count, w8 + L.partials, eA, eB, n_groups(p.D, p.group), p.group, p.D, p.w,
        reinterpret_cast<const int32_t *>(w8 + L.outtab));
}

template <int MW>
int combine_nl_small(const BInfo *info, const BHeader *hdr, const mw_batch &b, const mw_plan &p,
                     uint8_t *w8, const Layout &L, cudaStream_t s, int bits);

template <int MW>
int combine_nl(const BInfo *info, const BHeader *hdr, const mw_batch &b, const mw_plan &p,
               uint8_t *w8, const Layout &L, cudaStream_t s) {
  const int bits = 64 + p.w * (p.D - 1) + 1;
  if constexpr (MW == 16) {          // at least 52 x 16 bits: 14 to 17 limbs
    if (bits <= 896) launch_combine_b<MW, 14>(info, hdr, b, p, w8, L, s);
    else if (bits <= 960) launch_combine_b<MW, 15>(info, hdr, b, p, w8, L, s);
    else if (bits <= 1024) launch_combine_b<MW, 16>(info, hdr, b, p, w8, L, s);
    else if (bits <= 1088) launch_combine_b<MW, 17>(info, hdr, b, p, w8, L, s);
    else return fail(MW_EUNSUPPORTED, "too many diagonals for the fusion");
    return cuda_fail(cudaGetLastError(), "batch combine launch");
  } else {
    return combine_nl_small<MW>(info, hdr, b, p, w8, L, s, bits);
  }
}

template <int MW>
int combine_nl_small(const BInfo *info, const BHeader *hdr, const mw_batch &b, const mw_plan &p,
                     uint8_t *w8, const Layout &L, cudaStream_t s, int bits) {
  if (bits <= 256) launch_combine_b<MW, 4>(info, hdr, b, p, w8, L, s);
  else if (bits <= 320) launch_combine_b<MW, 5>(info, hdr, b, p, w8, L, s);
  else if (bits <= 384) launch_combine_b<MW, 6>(info, hdr, b, p, w8, L, s);
  else if (bits <= 448) launch_combine_b<MW, 7>(info, hdr, b, p, w8, L, s);
  else if (bits <= 512) launch_combine_b<MW, 8>(info, hdr, b, p, w8, L, s);
  else if (bits <= 576) launch_combine_b<MW, 9>(info, hdr, b, p, w8, L, s);
  else if (bits <= 640) launch_combine_b<MW, 10>(info, hdr, b, p, w8, L, s);
  else return fail(MW_EUNSUPPORTED, "too many diagonals for the fusion");
  return cuda_fail(cudaGetLastError(), "batch combine launch");
}

}  // namespace
}  // namespace mw

using namespace mw;

extern "C" {

int mw_batch_describe(int count, const int64_t *shapes, mw_batch *batch) {
  if (!shapes || !batch || count < 1) return fail(MW_EINVAL, "bad batch description");
  mw_batch b{};
  b.count = count;
  b.min_K = INT64_MAX;
  for (int i = 0; i < count; ++i) {
    const int64_t M = shapes[3 * i], N = shapes[3 * i + 1], K = shapes[3 * i + 2];
    if (M < 1 || N < 1 || K < 1) return fail(MW_EINVAL, "problem %d has an empty dimension", i);
    b.sum_M += M;
    b.sum_N += N;
    b.sum_MN += M * N;
    b.max_M = std::max(b.max_M, M);
    b.max_N = std::max(b.max_N, N);
    b.min_K = std::min(b.min_K, K);
    b.max_K = std::max(b.max_K, K);
  }
  *batch = b;
  return MW_OK;
}

int mw_gemm_batched_workspace_size(const mw_plan *plan, const mw_batch *batch, size_t *bytes) {
  if (!bytes) return fail(MW_EINVAL, "bytes is NULL");
  int rc = check_batch(plan, batch);
  if (rc) return rc;
  *bytes = layout_of(*plan, *batch).total;
  return MW_OK;
}

// The plan the spread measurement runs with: one piece, exponents only.
static mw_plan spread_plan(int m) {
  mw_plan p{};
  p.m = m; p.mode = MW_OZAKI; p.w = 8; p.S_A = p.S_B = 1; p.D = 1; p.group = 1; p.chunk = 64;
  p.range_A = p.range_B = -1;
  return p;
}

int mw_measure_spread_batched_workspace_size(int m, const mw_batch *batch, size_t *bytes) {
  if (!bytes) return fail(MW_EINVAL, "bytes is NULL");
  const mw_plan p = spread_plan(m);
  int rc = check_batch(&p, batch);
  if (rc) return rc;
  *bytes = layout_of(p, *batch).pieceA;
  return MW_OK;
}

int mw_measure_spread_batched(int m, const mw_batch *batch, const mw_problem *problems, void *ws,
                              size_t ws_bytes, int *range_A, int *range_B, mw_stream_t stream) {
  if (!range_A || !range_B || !problems) return fail(MW_EINVAL, "NULL argument");
  const mw_plan p = spread_plan(m);
  int rc = check_batch(&p, batch);
  if (rc) return rc;
  Layout L = layout_of(p, *batch);
  if (!ws || ws_bytes < L.pieceA) return fail(MW_ENOSPC, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = run_front(p, *batch, problems, ws, L, 1, s))) return rc;
  int32_t host[2];
  BHeader *hdr = reinterpret_cast<BHeader *>(static_cast<uint8_t *>(ws) + L.header);
  cudaError_t e = cudaMemcpyAsync(host, hdr->max_spread, sizeof host, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "batched spread read");
  *range_A = host[0];
  *range_B = host[1];
  return MW_OK;
}

int mw_gemm_batched(const mw_plan *plan, const mw_batch *batch, const mw_problem *problems,
                    void *ws, size_t ws_bytes, mw_stream_t stream) {
  int rc = check_batch(plan, batch);
  if (rc) return rc;
  if (!problems) return fail(MW_EINVAL, "problems is NULL");
  const mw_plan &p = *plan;
  const mw_batch &b = *batch;
  const Layout L = layout_of(p, b);
  if (!ws || ws_bytes < L.total)
    return fail(MW_ENOSPC, "workspace %zu bytes, need %zu", ws_bytes, L.total);
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t *w8 = static_cast<uint8_t *>(ws);
  phase(0, s);
  if ((rc = run_front(p, b, problems, ws, L, 0, s))) return rc;
  phase(1, s);
  ProductLaunch P{};
  P.pieceA = w8 + L.pieceA; P.pieceB = w8 + L.pieceB;
  P.rowsA = (int64_t)(L.packed ? 1 : p.S_A) * b.sum_M; P.rowsB = L.rowsB;
  P.Kpitch = L.Kpitch; P.KpitchB = L.KpitchB;
  P.S_A = p.S_A; P.S_B = p.S_B; P.D = p.D; P.w = p.w; P.group = L.sched; P.chunk = p.chunk;
  P.info = w8 + L.info; P.hdr = w8 + L.header; P.count = b.count;
  P.item_problem = reinterpret_cast<const int32_t *>(w8 + L.items);
  P.partials = w8 + L.partials;
  P.narrow = L.narrow;
  P.next_item = &reinterpret_cast<BHeader *>(w8 + L.header)->next_item;
  if ((rc = launch_product(P, s))) return rc;
  phase(2, s);
  const BInfo *info = reinterpret_cast<const BInfo *>(w8 + L.info);
  const BHeader *hdr = reinterpret_cast<const BHeader *>(w8 + L.header);
  switch (p.m) {
    case 2: rc = combine_nl<2>(info, hdr, b, p, w8, L, s); break;
    case 4: rc = combine_nl<4>(info, hdr, b, p, w8, L, s); break;
    case 8: rc = combine_nl<8>(info, hdr, b, p, w8, L, s); break;
    default: rc = combine_nl<16>(info, hdr, b, p, w8, L, s); break;
  }
  phase(3, s);
  return rc;
}

}  // extern "C"
