// MW_OZAKI: step 3 of the error-free summation on the tcgen05 tensor cores,
// step 4 as exact integer fusion.
//
// Section 4 observes that the diagonal convolutions s_i turn an m-double inner
// product into matrix products of pieces, "in particular tensor cores", the
// Ozaki scheme of Section 1.  Pieces are balanced integers |d| <= 2^(w-1),
// w <= 8, stored in bfloat16 (exact); a product of two pieces is at most
// 2^(2w-2) and a sum of `chunk` of them is at most 2^24, so the fp32
// accumulators of the tensor core hold exact integers.  After every chunk the
// accumulator is drained from tensor memory into integer registers (drain_parts2):
//   v = 4096 q + lo with q = round(v / 4096) by one fma against 1.5*2^23 and
//   lo = v - 4096 q exact (|lo| <= 2048); the bit patterns 0x4B400000 + q and
//   0x4B400000 + lo are joined as 4096 (0x4B400000 + q) + (0x4B400000 + lo) and
//   added as an unsigned value; the constant times the number of chunks is
//   subtracted at the end.
// Narrow mode (every s_t fits in int32): each diagonal sum is accumulated mod
// 2^32 and stored as an int32 plane.  Wide mode: a group of diagonals t0..t1
// is accumulated by Horner's rule mod 2^64, V = sum_t s_t 2^(w (t1 - t)), and
// stored as an int64 plane.  Planes are column-major per problem.  The fusion
// adds the planes exactly into one integer X and rounds X 2^(E_i + E_j + 4 -
// w(D+1)) to nearest into m words, one after the other (greedy); that fusion
// kernel is in mw_combine.cu.
//
// Product kernel (persistent, one CTA per SM; a work item is one output tile of
// one diagonal group):
//   warp 0      scheduler and TMA producer: takes work items from a global
//               counter in index order and hands them to the other roles
//               through a small ring in shared memory; per pipeline stage a
//               128 x 64 box of A_p and up to 256 x 64 of B_q (box heights in
//               steps of 16 rows, as many as the tile has)
//   warp 1      tensor-memory allocation and the single MMA-issuing thread
//   warps 2..   drain: warp w reads TMEM lanes 32 (w % 4).. and its share of columns
// Tiles are 128 x 256 (single products with N >= 256, and batches) or 128 x 128.
// Batches of small products (N <= 128) put rs = floor(256 / N) B slices of a
// problem side by side in one MMA: column block j of the accumulator is then
// diagonal t + j (zero slices before and after the B slices keep every block
// exact).  The same kernel serves one product (problem given in the launch
// parameters) and batches (device array of problems, mw_batched.cu).  Every wait
// is bounded.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "mw_device.cuh"
#include "mw_tc.cuh"
#include "mw_work.cuh"

namespace mw {
namespace {

#ifndef MW_WIDE_TILE
#define MW_WIDE_TILE 1   // 0: always 128 x 128 tiles (build knob for comparisons)
#endif
constexpr int BM = 128, BK = 64;
constexpr uint32_t STAGE_A = BM * BK * 2;
constexpr uint32_t MAGIC_BITS = 0x4B400000u;  // bit pattern of 1.5 * 2^23
constexpr uint64_t DRAIN_BIAS = (uint64_t)MAGIC_BITS * 4097u;   // what a drained value carries

// Packed fp32 arithmetic, two values per instruction (fma / add .f32x2: each
// element rounded as the scalar operation would round it).
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_pack(uint32_t lo, uint32_t hi) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(lo), "r"(hi));
  return d;
}
__device__ __forceinline__ void f2_unpack(uint64_t d, uint32_t &lo, uint32_t &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(d));
}
constexpr uint64_t kF2Magic = 0x4B4000004B400000ull;      // 1.5 2^23 twice
constexpr uint64_t kF2NegMagic = 0xCB400000CB400000ull;   // -1.5 2^23
constexpr uint64_t kF2Inv4096 = 0x3980000039800000ull;    // 2^-12
constexpr uint64_t kF2Neg4096 = 0xC5800000C5800000ull;    // -2^12

// An integer |v| <= 2^24 held exactly in fp32 as 4096 q + lo: h = 1.5 2^23 +
// round(v / 4096) (one rounding: v / 4096 is exact), lo = v - 4096 q exact; hb and
// lb are the bit patterns of 1.5 2^23 + q and 1.5 2^23 + lo, so that
// 4096 hb + lb = v + DRAIN_BIAS.  Two values v0, v1 at a time: hb and lb of
// each packed, v0's in the low half.
__device__ __forceinline__ void drain_parts2(uint32_t v0, uint32_t v1, uint64_t &hb,
                                             uint64_t &lb) {
  const uint64_t v = f2_pack(v0, v1);
  hb = f2_fma(v, kF2Inv4096, kF2Magic);
  lb = f2_add(f2_fma(f2_add(hb, kF2NegMagic), kF2Neg4096, v), kF2Magic);
}
// Kernel shapes.  Tile 128 x BN (BN = 128 or 256); NBUF accumulators of BN fp32
// columns in tensor memory (all 512 columns: with 128-column tiles four, so that
// the MMAs of short products run up to three drains ahead).  Two drain modes.  Narrow: every diagonal sum s_t
// fits in int32 (checked by the host), each diagonal is accumulated in 32-bit
// registers (arithmetic mod 2^32) and stored as int32.  Wide: a group of
// diagonals is accumulated by Horner's rule in int64 (BN = 128 only).
template <int BN_, bool NARROW> struct Shape {
  static constexpr int BN = BN_;
  static constexpr int STAGES = BN == 256 ? 4 : 6;            // 48 KB / 32 KB per stage
  static constexpr uint32_t STAGE_B = BN * BK * 2;
  static constexpr int WARPS = (NARROW && BN == 128) ? 16 : 8;  // drain warps
  static constexpr int COLS = BN * 4 / WARPS;                 // columns per drain thread
  static constexpr int THREADS = 64 + 32 * WARPS;
  static constexpr int NBUF = 512 / BN;
  static constexpr int TMEM_COLS = NBUF * BN;
  static constexpr size_t SMEM = 1024 + STAGES * (STAGE_A + STAGE_B) + 512;
  static_assert(NARROW || BN == 128, "wide drain only with 128-column tiles");
  static_assert(TMEM_COLS <= 512, "tensor memory holds 512 columns");
};
// Residue form, 128 x 256 tiles: a 4 KB box (32 rows x 64 residues, 128-byte
// swizzle) per drain warp, from which a tensor store writes the tile's residues.
template <int BN, bool CRT>
__host__ __device__ constexpr uint32_t out_stage_bytes() {
  return (CRT && BN == 256) ? (uint32_t)Shape<256, true>::WARPS * 4096u : 0u;
}
template <int BN, bool NARROW, bool CRT>
__host__ __device__ constexpr size_t kernel_smem() {
  return Shape<BN, NARROW>::SMEM + out_stage_bytes<BN, CRT>();
}
static_assert(kernel_smem<256, true, true>() <= 232448, "shared memory of one CTA");

constexpr int MAX_GROUPS = 128;
static_assert(MAX_GROUPS >= kCrtMaxModuli, "a work item per modulus");
// Residue form: drains between two reductions of the int32 accumulators mod p.
// A drain adds at most 2^24 in magnitude, so 127 of them (and a residue) stay
// below 2^31 - 2^24.
constexpr int kCrtReduceEvery = 127;
constexpr int RING = 4;   // work items the producer may run ahead

struct PParams {
  const BInfo *info;      // device array of problems, or nullptr: the one problem `single`
  const BHeader *hdr;     // totals (batched) or nullptr
  const int32_t *item_problem;  // batched: the problem of every work item
  int count;
  int S_A, S_B, D, w, group, G, chunk_kb;
  int64_t single_work;    // work items of `single`
  void *partials;         // int32 [t][M][N] (narrow) or int64 [g][M][N] (wide)
  unsigned long long *next_item;  // work counter, zero before the launch
  unsigned int *status;
  int gorder[MAX_GROUPS]; // diagonal groups, most expensive first
  // residue form: per modulus t, k-blocks per drain, the modulus, floor(2^32 / p),
  // the offset B_t >= 2^31 with B_t = (p - 1) / 2 mod p, and 1.5 2^23 + (p - 1) / 2
  uint8_t crt_chunk_kb[MAX_GROUPS];
  uint16_t crt_p[MAX_GROUPS];
  uint32_t crt_m32[MAX_GROUPS], crt_off[MAX_GROUPS];
  float crt_cf[MAX_GROUPS];
  BInfo single;
};

// Tensor maps over the two piece arrays with boxes of 16, 32, ..., 256 rows (A)
// and 8, 16, ..., 256 rows (B): a tile loads only the rows its problem has,
// rounded up (rows past them would only feed outputs that are never stored).
// The residue form with 128 x 256 tiles also stores through a map (`out`: the
// residue planes, boxes of 64 columns x 32 rows).  6 KB of kernel parameters.
constexpr int NBOX = 16, NBOXB = 32;
struct Maps {
  CUtensorMap a[NBOX], b[NBOXB], out;
};
__host__ __device__ constexpr int box_rows(int i) { return 16 * (i + 1); }
__device__ __forceinline__ int box_index(int64_t rows) {
  return rows <= 16 ? 0 : rows >= 256 ? NBOX - 1 : (int)((rows + 15) >> 4) - 1;
}
// B boxes in steps of 8 rows: a stacked block of N8 rows starts on a swizzle atom
__host__ __device__ constexpr int box_rows_b(int i) { return 8 * (i + 1); }
__device__ __forceinline__ int box_index_b(int64_t rows) {
  return rows <= 8 ? 0 : rows >= 256 ? NBOXB - 1 : (int)((rows + 7) >> 3) - 1;
}

__device__ __forceinline__ const BInfo &problem(const PParams &P, int i) {
  return P.info ? P.info[i] : P.single;
}

struct Item {
  int i, g, t0, t1, tm, tn, KB, rs, K8, Z, N8;
  int64_t M, N, rowA, rowB, part;
};

// Work item u: problem, output tile, diagonals t0..t1.  Single products take
// the diagonal groups most expensive first (gorder); a batch's problems carry
// their own diagonals per item (nd) and items per tile (G).
__device__ __forceinline__ Item decode_item(const PParams &P, int64_t u) {
  Item x;
  x.i = P.item_problem ? P.item_problem[u]
      : P.info ? find_problem(P.info, P.count, u, [](const BInfo &b) { return b.work; }) : 0;
  const BInfo &b = problem(P, x.i);
  const int64_t local = u - b.work;
  const int tiles = b.tiles_m * b.tiles_n;
  const int tile = (int)(local % tiles);
  x.tm = tile % b.tiles_m;
  x.tn = tile / b.tiles_m;
  const int nd = P.info ? b.nd : P.group;
  x.g = P.info ? (int)(local / tiles) : P.gorder[(int)(local / tiles)];
  x.t0 = x.g * nd;
  x.t1 = min(P.D, x.t0 + nd) - 1;
  x.rs = P.info ? b.rs : 1;
  x.KB = b.KB;
  x.K8 = b.K8; x.Z = b.Z; x.N8 = (int)((b.N + 7) & ~(int64_t)7);
  x.M = b.M; x.N = b.N; x.rowA = b.rowA; x.rowB = b.rowB; x.part = b.part;
  return x;
}
// A block of rs diagonals t..t+rs-1 sweeps the A slices p = plo..phi against
// the rs B slices t-p .. t-p+rs-1 (zero slices outside 0..S_B-1): column block
// j collects exactly the pairs of diagonal t + j.
__device__ __forceinline__ int plo(const PParams &P, int t) { return max(0, t - P.S_B + 1); }
__device__ __forceinline__ int phi(const PParams &P, int t, int rs) {
  return min(t + rs - 1, P.S_A - 1);
}
__device__ __forceinline__ int nsteps(const PParams &P, int t, int rs, int KB) {
  const int n = phi(P, t, rs) - plo(P, t) + 1;
  return n > 0 ? n * KB : 0;
}

// The pairs of "diagonal" t and their k-blocks: the slice form sweeps
// p = plo..phi against B slice t - p; the residue form (CRT) has one pair per
// modulus t, residue plane t of A against residue plane t of B.
template <bool CRT>
__device__ __forceinline__ int pair_lo(const PParams &P, int t) { return CRT ? t : plo(P, t); }
template <bool CRT>
__device__ __forceinline__ int pair_hi(const PParams &P, int t, int rs) {
  return CRT ? t : phi(P, t, rs);
}
template <bool CRT>
__device__ __forceinline__ int steps_of(const PParams &P, int t, int rs, int KB) {
  return CRT ? KB : nsteps(P, t, rs, KB);
}
template <bool CRT>
__device__ __forceinline__ int chunk_of(const PParams &P, int t) {
  return CRT ? (int)P.crt_chunk_kb[t] : P.chunk_kb;
}
// K-packed batches: the pairs of the block of diagonals t..t+rs-1 are one
// contiguous contraction over A columns plo K8 .. (phi + 1) K8 (the B columns move
// with them; overhangs read zeros), in 64-wide k-blocks
__device__ __forceinline__ int kp_steps(const PParams &P, const Item &x, int t) {
  const int n = phi(P, t, x.rs) - plo(P, t) + 1;
  return n > 0 ? (n * x.K8 + BK - 1) / BK : 0;
}
template <bool STACK, bool CRT>
__device__ __forceinline__ int item_steps(const PParams &P, const Item &x, int t) {
  if constexpr (STACK) return kp_steps(P, x, t);
  else return steps_of<CRT>(P, t, x.rs, x.KB);
}

// STACK: B slices side by side (batches of small products); otherwise one
// slice per MMA and the drain stores one diagonal per tile column.
// CRT: the residue form, one product of residue planes per modulus (narrow,
// not stacked); its int32 sums are reduced mod p every kCrtReduceEvery drains,
// so they stay congruent to the exact sums for any K.
template <int BN_, bool NARROW, bool STACK, bool CRT = false>
__global__ void __launch_bounds__(Shape<BN_, NARROW>::THREADS, 1)
    ozaki_kernel(const __grid_constant__ Maps maps, const PParams P) {
  static_assert(!CRT || (NARROW && !STACK), "the residue form is narrow, one product per item");
  using SH = Shape<BN_, NARROW>;
  constexpr int BN = SH::BN, STAGES = SH::STAGES, TMEM_COLS = SH::TMEM_COLS;
  constexpr uint32_t STAGE_B = SH::STAGE_B;
  constexpr int NUM_DRAIN_WARPS = SH::WARPS;
  constexpr int NBUF = SH::NBUF;
  constexpr bool OUT_TMA = out_stage_bytes<BN, CRT>() > 0;

  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * STAGE_A;
  uint8_t *sOut = smem + STAGES * (STAGE_A + STAGE_B);   // 1024-byte aligned
  uint64_t *full = (uint64_t *)(sOut + out_stage_bytes<BN, CRT>());
  uint64_t *empty = full + STAGES;
  uint64_t *accf = empty + STAGES;
  uint64_t *acce = accf + NBUF;
  uint64_t *done = acce + NBUF;
  uint64_t *uf = done + 1;           // work item published
  uint64_t *ue = uf + RING;          // work item read by the MMA thread and every drain warp
  volatile int64_t *ring = (volatile int64_t *)(ue + RING);
  uint32_t *tmem_holder = (uint32_t *)(ring + RING);
  volatile int *abort = (volatile int *)(tmem_holder + 1);
  int *counters = (int *)(tmem_holder + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t total = P.hdr ? (P.hdr->bad ? 0 : P.hdr->total_work) : P.single_work;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], NUM_DRAIN_WARPS);
    }
    mbar_init(done, 1);
    for (int r = 0; r < RING; ++r) {
      mbar_init(&uf[r], 1);
      mbar_init(&ue[r], 1 + NUM_DRAIN_WARPS);
    }
    *abort = 0;
    counters[0] = counters[1] = 0;
    fence_barrier_init();
    for (int i = 0; i < NBOX; ++i) prefetch_map(&maps.a[i]);
    for (int i = 0; i < NBOXB; ++i) prefetch_map(&maps.b[i]);
    if constexpr (OUT_TMA) prefetch_map(&maps.out);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      // dynamic schedule: items in index order (largest first) from a global counter,
      // published to the other roles through a ring of RING slots
      for (uint32_t k = 0; !*abort; ++k) {
        const uint32_t slot = k % RING, rph = (k / RING) & 1;
        const int64_t got = (int64_t)atomicAdd(P.next_item, 1ull);
        if (!mbar_wait(&ue[slot], rph ^ 1, P.status, abort)) break;
        const int64_t u = got < total ? got : -1;
        ring[slot] = u;
        mbar_arrive(&uf[slot]);
        if (u < 0) break;
        Item x = decode_item(P, u);
        if constexpr (!STACK) x.rs = 1;
        const int ia = box_index(min((int64_t)BM, x.M - (int64_t)x.tm * BM));
        // stacked batches: one box of N8 rows per column block; otherwise one box
        const int brows = (STACK && x.rs > 1) ? x.N8
                                              : (int)min((int64_t)BN, x.rs * x.N - (int64_t)x.tn * BN);
        const int ib = box_index_b(brows);
        const int nbox = STACK ? x.rs : 1;
        // the boxes of maps.a are at most BM rows and of maps.b at most BN rows
        const uint32_t bytes =
            (uint32_t)(min(box_rows(ia), BM) + nbox * min(box_rows_b(ib), BN)) * BK * 2;
        for (int t = x.t0; t <= x.t1 && !*abort; t += x.rs) {
          if constexpr (STACK) {
            // A columns plo K8 + 64 kb; column block jb (diagonal t + jb) reads B at
            // (Z + S_B - 1 - t - jb) K8 further on: slice q = t + jb - p meets slice p
            const int64_t k0 = (int64_t)plo(P, t) * x.K8;
            const int64_t xb = k0 + (int64_t)(x.Z + P.S_B - 1 - t) * x.K8;
            const int ra = (int)(x.rowA + (int64_t)x.tm * BM);
            const int rb = (int)(x.rowB + (int64_t)x.tn * BN);
            const int nst = kp_steps(P, x, t);
            for (int kb = 0; kb < nst; ++kb, ++it) {
              const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
              if (!mbar_wait(&empty[s], ph ^ 1, P.status, abort)) break;
              mbar_arrive_expect_tx(&full[s], bytes);
              tma_load_2d(smem_u32(sA + s * STAGE_A), &maps.a[ia], (int)(k0 + kb * BK), ra,
                          smem_u32(&full[s]));
              for (int jb = 0; jb < x.rs; ++jb)
                tma_load_2d(smem_u32(sB + s * STAGE_B + (uint32_t)(jb * x.N8) * (BK * 2)),
                            &maps.b[ib], (int)(xb - (int64_t)jb * x.K8 + kb * BK), rb,
                            smem_u32(&full[s]));
              counters[0] = (int)it + 1;
            }
          } else {
            for (int p = pair_lo<CRT>(P, t); p <= pair_hi<CRT>(P, t, x.rs) && !*abort; ++p) {
              const int q = CRT ? t : t - p;        // first of the rs B slices
              const int ra = (int)(x.rowA + (int64_t)p * x.M + (int64_t)x.tm * BM);
              const int rb = (int)(x.rowB + (int64_t)(q + x.rs - 1) * x.N + (int64_t)x.tn * BN);
              for (int kb = 0; kb < x.KB; ++kb, ++it) {
                const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1, P.status, abort)) break;
                mbar_arrive_expect_tx(&full[s], bytes);
                tma_load_2d(smem_u32(sA + s * STAGE_A), &maps.a[ia], kb * BK, ra,
                            smem_u32(&full[s]));
                tma_load_2d(smem_u32(sB + s * STAGE_B), &maps.b[ib], kb * BK, rb,
                            smem_u32(&full[s]));
                counters[0] = (int)it + 1;
              }
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      uint32_t it = 0, ch = 0;
      for (uint32_t k = 0; !*abort; ++k) {
        const uint32_t slot = k % RING, rph = (k / RING) & 1;
        if (!mbar_wait(&uf[slot], rph, P.status, abort)) break;
        const int64_t u = ring[slot];
        mbar_arrive(&ue[slot]);
        if (u < 0) break;
        Item x = decode_item(P, u);
        if constexpr (!STACK) x.rs = 1;
        // N of the MMA: the tile's valid columns rounded up to 16
        const int ncols = (STACK && x.rs > 1) ? x.rs * x.N8
                                              : (int)min((int64_t)BN, x.rs * x.N - (int64_t)x.tn * BN);
        const uint32_t idesc = idesc_bf16(BM, (ncols + 15) & ~15);
        for (int t = x.t0; t <= x.t1 && !*abort; t += x.rs) {
          const int tot = item_steps<STACK, CRT>(P, x, t);
          const int ck = chunk_of<CRT>(P, t);
          for (int j = 0; j < tot && !*abort; ++ch) {
            const int nk = min(ck, tot - j);
            const uint32_t b = ch % NBUF, bph = (ch / NBUF) & 1;
            if (!mbar_wait(&acce[b], bph ^ 1, P.status, abort)) break;
            tc_fence_after();
            const uint32_t d = tmem + b * BN;
            for (int jj = 0; jj < nk; ++jj, ++it) {
              const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
              if (!mbar_wait(&full[s], ph, P.status, abort)) break;
              tc_fence_after();
              const uint64_t ad = sw128_desc(smem_u32(sA + s * STAGE_A));
              const uint64_t bd = sw128_desc(smem_u32(sB + s * STAGE_B));
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                tc_mma(d, ad + 2 * kk, bd + 2 * kk, idesc, (jj | kk) ? 1u : 0u);
              tc_commit(&empty[s]);
              counters[1] = (int)it + 1;
            }
            tc_commit(&accf[b]);
            j += nk;
          }
        }
      }
      tc_commit(done);
      volatile int never = 0;
      mbar_wait(done, 0, P.status, &never);
    }
  } else {
    constexpr int COLS = SH::COLS;
    const int quarter = warp & 3;                 // TMEM lanes this warp may read
    const int slice = (warp - 2) >> 2;            // which COLS columns of the tile
    const int row = quarter * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + slice * COLS;
    uint32_t ch = 0;
    bool ok = true;
    for (uint32_t k = 0; ok; ++k) {
      const uint32_t slot = k % RING, rph = (k / RING) & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(&uf[slot], rph, P.status, abort))) break;
      const int64_t u = ring[slot];
      __syncwarp();
      if (lane == 0) mbar_arrive(&ue[slot]);
      if (u < 0) break;
      Item x = decode_item(P, u);
      if constexpr (!STACK) x.rs = 1;
      const int64_t r = (int64_t)x.tm * BM + row;
      const int64_t c0 = (int64_t)x.tn * BN + slice * COLS;
      if constexpr (NARROW) {
        // one block of rs diagonals at a time in 32-bit accumulators, stored as
        // int32 s_t; column c of the tile is column c mod N of diagonal t + c / N
        for (int t = x.t0; t <= x.t1 && ok; t += x.rs) {
          uint32_t acc[COLS];
#pragma unroll
          for (int i = 0; i < COLS; ++i) acc[i] = 0;
          const int ck = chunk_of<CRT>(P, t);
          const int nch = (item_steps<STACK, CRT>(P, x, t) + ck - 1) / ck;
          int since = 0;                          // drains since the last reduction
          for (int c = 0; c < nch; ++c, ++ch) {
            const uint32_t b = ch % NBUF, bph = (ch / NBUF) & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&accf[b], bph, P.status, abort))) {
              ok = false;
              break;
            }
            tc_fence_after();
            // 16 columns per load: with 32 the accumulators and the loaded values
            // no longer fit in the registers of a thread (10 warps per CTA)
#pragma unroll
            for (int h = 0; h < COLS / 16; ++h) {
              uint32_t v[16];
              tc_ld16(tbase + b * BN + 16 * h, v);
              tc_wait_ld();
              if (h == COLS / 16 - 1) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[b]);
              }
#pragma unroll
              for (int i = 0; i < 16; i += 2) {
                uint64_t hb, lb;
                drain_parts2(v[i], v[i + 1], hb, lb);
                uint32_t h0, h1, l0, l1;
                f2_unpack(hb, h0, h1);
                f2_unpack(lb, l0, l1);
                acc[16 * h + i] += (h0 << 12) + l0;
                acc[16 * h + i + 1] += (h1 << 12) + l1;
              }
            }
            ++since;
            if constexpr (CRT) {
              if (since == kCrtReduceEvery && c + 1 < nch) {
                const int pm = P.crt_p[t];
                const uint32_t bs = (uint32_t)since * (uint32_t)DRAIN_BIAS;
#pragma unroll
                for (int i = 0; i < COLS; ++i) acc[i] = (uint32_t)((int32_t)(acc[i] - bs) % pm);
                since = 0;
              }
            }
          }
          if (!ok) break;
          if constexpr (OUT_TMA) {
            // the balanced residues (see below) in pairs, column 2e in the low half;
            // the warp writes them box by box into its staging box, one tensor store
            // each (rows past M and columns past N are not written)
            const uint32_t pm = P.crt_p[t], m32 = P.crt_m32[t];
            const uint32_t offb = P.crt_off[t] - (uint32_t)since * (uint32_t)DRAIN_BIAS;
            const float cf = P.crt_cf[t];
            const uint64_t ncf = f2_pack(__float_as_uint(-cf), __float_as_uint(-cf));
            uint32_t pk[COLS / 2];
#pragma unroll
            for (int e = 0; e < COLS / 2; ++e) {
              uint32_t rb[2];
#pragma unroll
              for (int o = 0; o < 2; ++o) {
                const uint32_t u = acc[2 * e + o] + offb;
                const uint32_t r0 = u - __umulhi(u, m32) * pm;
                rb[o] = 0x4B400000u + min(r0, r0 - pm);
              }
              uint32_t f0, f1;
              f2_unpack(f2_add(f2_pack(rb[0], rb[1]), ncf), f0, f1);
              asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(pk[e]) : "r"(f0), "r"(f1));
            }
            uint8_t *box = sOut + (warp - 2) * 4096;
            const int y = (int)((int64_t)x.tm * BM + quarter * 32);
#pragma unroll
            for (int hf = 0; hf < COLS / 64; ++hf) {
              if (lane == 0) bulk_wait_read();     // the box's previous store has read it
              __syncwarp();
#pragma unroll
              for (int g = 0; g < 8; ++g)
                *reinterpret_cast<uint4 *>(box + lane * 128 + ((g ^ (lane & 7)) << 4)) =
                    make_uint4(pk[32 * hf + 4 * g], pk[32 * hf + 4 * g + 1],
                               pk[32 * hf + 4 * g + 2], pk[32 * hf + 4 * g + 3]);
              fence_proxy_async_smem();
              __syncwarp();
              if (lane == 0 && y < x.M && c0 + 64 * hf < x.N)
                tma_store_3d(&maps.out, (int)(c0 + 64 * hf), y, t, smem_u32(box));
            }
          } else if (r < x.M) {
            // planes are column-major: lanes (consecutive rows) store consecutive words
            const uint32_t bias = (uint32_t)since * (uint32_t)DRAIN_BIAS;
            if constexpr (STACK) {
              // column block j (diagonal t + j) is N8 columns wide when stacked
              const int nd = min(x.rs, x.t1 - t + 1);     // diagonals of this block to keep
              const int64_t nw = x.rs > 1 ? x.N8 : x.N;
              int j = (int)(c0 / nw);
              int64_t col = c0 - (int64_t)j * nw;
              int32_t *base = static_cast<int32_t *>(P.partials) + x.part + r;
#pragma unroll
              for (int i = 0; i < COLS; ++i) {
                if (j < nd && col < x.N)
                  base[((int64_t)(t + j) * x.N + col) * x.M] = (int32_t)(acc[i] - bias);
                if (++col == nw) {
                  col = 0;
                  ++j;
                }
              }
            } else if constexpr (CRT) {
              // the balanced residue of each sum S, as bfloat16 (|r| <= 256): with
              // u = S + B_t in [0, 2^32) (|S| < 2^31 - 2^24 + p), u mod p by the
              // reciprocal (the quotient estimate is exact or one short), then
              // r = u mod p - (p - 1) / 2 as a float from its bits.  The row's
              // COLS residues are contiguous: 16-byte stores of eight
              const uint32_t pm = P.crt_p[t], m32 = P.crt_m32[t], off = P.crt_off[t];
              const float cf = P.crt_cf[t];
              auto resid = [&](uint32_t a) -> uint32_t {   // bf16 bits in the high half
                const uint32_t u = a - bias + off;
                const uint32_t r0 = u - __umulhi(u, m32) * pm;
                const uint32_t rr = min(r0, r0 - pm);
                return __float_as_uint(__uint_as_float(0x4B400000u + rr) - cf);
              };
              uint16_t *dst = static_cast<uint16_t *>(P.partials) +
                              ((int64_t)t * x.M + r) * crt_ld(x.N) + c0;
              if (c0 + COLS <= x.N) {
#pragma unroll
                for (int g = 0; g < COLS / 8; ++g) {
                  uint32_t w[4];
#pragma unroll
                  for (int e = 0; e < 4; ++e)
                    asm("prmt.b32 %0, %1, %2, 0x7632;"
                        : "=r"(w[e])
                        : "r"(resid(acc[8 * g + 2 * e])), "r"(resid(acc[8 * g + 2 * e + 1])));
                  *reinterpret_cast<uint4 *>(dst + 8 * g) = make_uint4(w[0], w[1], w[2], w[3]);
                }
              } else {
#pragma unroll
                for (int i = 0; i < COLS; ++i)
                  if (c0 + i < x.N) dst[i] = (uint16_t)(resid(acc[i]) >> 16);
              }
            } else {
              int32_t *dst = static_cast<int32_t *>(P.partials) + x.part + (int64_t)t * x.N * x.M + r;
#pragma unroll
              for (int i = 0; i < COLS; ++i)
                if (c0 + i < x.N) dst[(c0 + i) * x.M] = (int32_t)(acc[i] - bias);
            }
          }
        }
      } else {
        uint64_t acc[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) acc[i] = 0;
        uint64_t bias = 0;
        for (int t = x.t0; t <= x.t1 && ok; ++t) {
          if (t > x.t0) {
#pragma unroll
            for (int i = 0; i < 64; ++i) acc[i] <<= P.w;
            bias <<= P.w;
          }
          const int nch = (nsteps(P, t, 1, x.KB) + P.chunk_kb - 1) / P.chunk_kb;
          bias += (uint64_t)nch * DRAIN_BIAS;
          for (int c = 0; c < nch; ++c, ++ch) {
            const uint32_t b = ch % NBUF, bph = (ch / NBUF) & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&accf[b], bph, P.status, abort))) {
              ok = false;
              break;
            }
            tc_fence_after();
            uint32_t v[32];
            tc_ld32(tbase + b * BN, v);
            tc_wait_ld();
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
              uint64_t hb, lb;
              drain_parts2(v[i], v[i + 1], hb, lb);
              acc[i] += ((uint64_t)(uint32_t)hb << 12) + (uint32_t)lb;
              acc[i + 1] += ((hb >> 32) << 12) + (lb >> 32);
            }
            tc_ld32(tbase + b * BN + 32, v);
            tc_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[b]);
#pragma unroll
            for (int i = 0; i < 32; i += 2) {
              uint64_t hb, lb;
              drain_parts2(v[i], v[i + 1], hb, lb);
              acc[32 + i] += ((uint64_t)(uint32_t)hb << 12) + (uint32_t)lb;
              acc[32 + i + 1] += ((hb >> 32) << 12) + (lb >> 32);
            }
          }
        }
        if (!ok) break;
        // the group's Horner sum, plane g column-major
        if (r < x.M) {
          int64_t *dst = static_cast<int64_t *>(P.partials) + x.part + (int64_t)x.g * x.N * x.M + r;
#pragma unroll
          for (int i = 0; i < 64; ++i)
            if (c0 + i < x.N) dst[(c0 + i) * x.M] = (int64_t)(acc[i] - bias);
        }
      }
    }
    if constexpr (OUT_TMA)
      if (lane == 0) bulk_wait_all();             // the residue stores are complete
  }

  __syncthreads();
  if (warp == 0 && lane == 0 && *abort) {
    for (int i = counters[1]; i < counters[0]; ++i) {
      volatile int never = 0;
      mbar_wait(&full[i % STAGES], (i / STAGES) & 1, P.status, (volatile int *)&never);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 2D map over a bf16 array of `rows` rows of `pitch` elements; boxes of 64 x 128,
// 128-byte swizzle (the layout sw128_desc describes).
int make_map_2d(CUtensorMap *map, const void *base, int64_t pitch, int64_t rows, int box_rows) {
  const uint64_t dims[2] = {(uint64_t)pitch, (uint64_t)rows};
  const uint64_t strides[1] = {(uint64_t)pitch * 2};
  const uint32_t box[2] = {BK, (uint32_t)box_rows};
  return make_map_bf16(map, base, 2, dims, strides, box);
}

}  // namespace

int make_map_bf16(void *map, const void *base, int rank, const uint64_t *dims,
                  const uint64_t *strides, const uint32_t *box, bool swizzle128) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  if (!fn) return fail(MW_ECUDA, "cuTensorMapEncodeTiled not available");
  if (rank < 1 || rank > 5) return fail(MW_EINVAL, "tensor map rank %d", rank);
  cuuint64_t d[5], st[4];
  cuuint32_t bx[5], estr[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    bx[i] = box[i];
    estr[i] = 1;
    if (i + 1 < rank) st[i] = strides[i];
  }
  CUresult r = fn(static_cast<CUtensorMap *>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank,
                  const_cast<void *>(base), d, st, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(MW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return MW_OK;
}

int launch_product(const ProductLaunch &a, cudaStream_t s) {
  const int G = n_groups(a.D, a.group);
  if (G > MAX_GROUPS) return fail(MW_EUNSUPPORTED, "more than %d diagonal groups", MAX_GROUPS);
  if (a.crt) {
    if (a.D > crt_table_size() || a.info || !a.narrow)
      return fail(MW_EINVAL, "residue form: single products, at most %d moduli", crt_table_size());
  } else {
    if (a.chunk < BK || a.chunk % BK)
      return fail(MW_EINVAL, "chunk must be a positive multiple of 64");
    if (a.w < 2 || a.w > 8 || (int64_t)a.chunk << (2 * a.w - 2) > (1 << 24))
      return fail(MW_EINVAL, "chunk * 2^(2w-2) must not exceed 2^24 (w=%d chunk=%d)", a.w,
                  a.chunk);
  }
  if (a.rowsA > 0x7fffffffLL || a.rowsB > 0x7fffffffLL)
    return fail(MW_EUNSUPPORTED, "more than 2^31 piece rows");
  // 128 x 256 tiles for a single wide product in narrow mode (half the A-operand
  // traffic per flop); batches of small products keep 128 x 128.
  const int bn = a.info ? (a.narrow ? 256 : 128)
                        : ((MW_WIDE_TILE && a.narrow && a.N >= 256) ? 256 : 128);
  PParams P{};
  P.info = static_cast<const BInfo *>(a.info);
  P.hdr = static_cast<const BHeader *>(a.hdr);
  P.item_problem = a.item_problem;
  P.count = a.count;
  P.S_A = a.S_A; P.S_B = a.S_B; P.D = a.D; P.w = a.w; P.group = a.group; P.G = G;
  P.chunk_kb = a.crt ? 1 : a.chunk / BK;
  if (a.crt)
    for (int t = 0; t < a.D; ++t) {
      const uint32_t p = (uint32_t)crt_modulus(t), h = (p - 1) / 2;
      P.crt_chunk_kb[t] = (uint8_t)(crt_chunk(t) / BK);
      P.crt_p[t] = (uint16_t)p;
      P.crt_m32[t] = (uint32_t)((1ull << 32) / p);
      P.crt_off[t] = (uint32_t)((1ull << 31) + (h + p - (uint32_t)((1ull << 31) % p)) % p);
      P.crt_cf[t] = 12582912.0f + (float)h;
    }
  P.partials = a.partials;
  P.next_item = a.next_item;
  P.status = status_ptr();
  if (!a.info) {
    BInfo &b = P.single;
    b.M = a.M; b.N = a.N; b.K = a.K;
    b.tiles_m = (int)((a.M + BM - 1) / BM);
    b.tiles_n = (int)((a.N + bn - 1) / bn);
    b.KB = (int)((a.K + BK - 1) / BK);
    b.rs = 1; b.nd = a.group; b.G = G;
    P.single_work = (int64_t)G * b.tiles_m * b.tiles_n;
  }
  // most expensive groups first: pairs on a diagonal grow, then shrink
  long long cost[MAX_GROUPS];
  for (int g = 0; g < G; ++g) {
    cost[g] = 0;
    for (int t = g * a.group; t < std::min(a.D, (g + 1) * a.group); ++t)
      cost[g] += a.crt ? 1 : std::max(0, std::min(t, a.S_A - 1) - std::max(0, t - a.S_B + 1) + 1);
    P.gorder[g] = g;
  }
  for (int i = 1; i < G; ++i)
    for (int j = i; j > 0 && cost[P.gorder[j]] > cost[P.gorder[j - 1]]; --j)
      std::swap(P.gorder[j], P.gorder[j - 1]);
  Maps maps;
  int rc = MW_OK;
  for (int i = 0; i < NBOX && !rc; ++i)
    rc = make_map_2d(&maps.a[i], a.pieceA, a.Kpitch, a.rowsA, std::min(box_rows(i), BM));
  for (int i = 0; i < NBOXB && !rc; ++i)
    rc = make_map_2d(&maps.b[i], a.pieceB, a.KpitchB, a.rowsB, std::min(box_rows_b(i), bn));
  if (!rc && a.crt && bn == 256) {
    // residue planes [t][i][j], rows of crt_ld(N) elements
    const uint64_t ld = (uint64_t)crt_ld(a.N);
    const uint64_t dims[3] = {(uint64_t)a.N, (uint64_t)a.M, (uint64_t)a.D};
    const uint64_t strides[2] = {ld * 2, ld * 2 * (uint64_t)a.M};
    const uint32_t box[3] = {64, 32, 1};
    rc = make_map_bf16(&maps.out, a.partials, 3, dims, strides, box);
  } else {
    memset(&maps.out, 0, sizeof maps.out);
  }
  if (rc) return rc;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(ozaki_kernel<128, true, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Shape<128, true>::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ozaki_kernel<128, false, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Shape<128, false>::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ozaki_kernel<256, true, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Shape<256, true>::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ozaki_kernel<256, true, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Shape<256, true>::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ozaki_kernel<256, true, false, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kernel_smem<256, true, true>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ozaki_kernel<128, true, false, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)Shape<128, true>::SMEM);
    if (e != cudaSuccess) return cuda_fail(e, "product kernel smem attribute");
    attr_set = true;
  }
  cudaError_t e = cudaMemsetAsync(a.next_item, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return cuda_fail(e, "work counter reset");
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int grid = nsm;
  if (!a.info) grid = (int)std::min<int64_t>(P.single_work, nsm);
  using S256 = Shape<256, true>;
  using S128 = Shape<128, true>;
  using W128 = Shape<128, false>;
  if (a.crt && bn == 256)
    ozaki_kernel<256, true, false, true><<<grid, S256::THREADS, kernel_smem<256, true, true>(), s>>>(
        maps, P);
  else if (a.crt)
    ozaki_kernel<128, true, false, true><<<grid, S128::THREADS, S128::SMEM, s>>>(maps, P);
  else if (a.narrow && bn == 256 && a.info)
    ozaki_kernel<256, true, true><<<grid, S256::THREADS, S256::SMEM, s>>>(maps, P);
  else if (a.narrow && bn == 256)
    ozaki_kernel<256, true, false><<<grid, S256::THREADS, S256::SMEM, s>>>(maps, P);
  else if (a.narrow)
    ozaki_kernel<128, true, false><<<grid, S128::THREADS, S128::SMEM, s>>>(maps, P);
  else
    ozaki_kernel<128, false, false><<<grid, W128::THREADS, W128::SMEM, s>>>(maps, P);
  return cuda_fail(cudaGetLastError(), "product kernel launch");
}

bool narrow_partials(int S_A, int S_B, int w, int64_t max_K) {
  const int64_t S_min = std::min(S_A, S_B);
  return (double)S_min * (double)max_K * std::ldexp(1.0, 2 * w - 2) < 2147483648.0;
}

size_t ozaki_partials_planes_bytes(int64_t M, int64_t N, int D, int group, bool narrow) {
  return (narrow ? (size_t)D * 4 : (size_t)n_groups(D, group) * 8) * M * N;
}

size_t crt_residue_planes_bytes(int64_t M, int64_t N, int D) {
  return (size_t)D * M * crt_ld(N) * 2;
}

size_t crt_partials_bytes(int64_t M, int64_t N, int D) {
  return ((crt_residue_planes_bytes(M, N, D) + 255) & ~(size_t)255) + 256;
}

size_t ozaki_partials_bytes(int64_t M, int64_t N, int D, int group, bool narrow) {
  // partial sums, then the 8-byte work counter at the next 256-byte boundary
  const size_t planes = ozaki_partials_planes_bytes(M, N, D, group, narrow);
  return ((planes + 255) & ~(size_t)255) + 256;
}

int launch_ozaki(const OzakiArgs &a, cudaStream_t s, const std::function<void()> &between_kernels) {
  if (a.Kp % BK) return fail(MW_EINVAL, "padded K must be a multiple of %d", BK);
  const int G = n_groups(a.D, a.group);
  // the residue form keeps one int32 sum per modulus (reduced mod p as it goes)
  const bool narrow = a.crt || narrow_partials(a.S_A, a.S_B, a.w, a.Kp);
  ProductLaunch L{};
  L.pieceA = a.dA; L.pieceB = a.dB;
  // rows the piece arrays hold: S_A / S_B digit planes, or D residue planes (the
  // tensor maps' extent, beyond which TMA fills zeros)
  L.rowsA = (int64_t)(a.crt ? a.D : a.S_A) * a.M;
  L.rowsB = (int64_t)(a.crt ? a.D : a.S_B) * a.N;
  L.Kpitch = L.KpitchB = a.Kp;
  L.S_A = a.S_A; L.S_B = a.S_B; L.D = a.D; L.w = a.w; L.chunk = a.chunk;
  L.group = a.crt ? 1 : sched_group(a.D, a.group, narrow);
  L.crt = a.crt;
  L.info = nullptr; L.hdr = nullptr; L.count = 1;
  L.M = a.M; L.N = a.N; L.K = a.Kp;
  L.partials = a.partials;
  L.narrow = narrow;
  const size_t planes = a.crt ? crt_residue_planes_bytes(a.M, a.N, a.D)
                              : ozaki_partials_planes_bytes(a.M, a.N, a.D, a.group, narrow);
  L.next_item = reinterpret_cast<unsigned long long *>(
      reinterpret_cast<uint8_t *>(a.partials) + ((planes + 255) & ~(size_t)255));
  int rc = launch_product(L, s);
  if (rc) return rc;
  if (between_kernels) between_kernels();
  return a.crt ? launch_crt_combine(a, s) : launch_combine(a, G, narrow, s);
}

}  // namespace mw
