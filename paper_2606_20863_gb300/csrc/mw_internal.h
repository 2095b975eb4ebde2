// Internal declarations of libmw shared by its translation units (not installed).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include <functional>

#include "../../include/mw.h"

namespace mw {

// Host-side error message of the calling thread (mw_last_error).
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// Device address of the status word of the current device.
unsigned int *status_ptr();

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// ---- split (mw_split.cu) ----------------------------------------------------
struct SplitArgs {
  int m, trans, w, S, format, range;
  int nmod;                     // residue form: moduli (planes), S = fixed-point bits; else 0
  int64_t R, K, ld, plane_stride, digit_ld;
  const double *X;
  void *digits;
  int32_t *exps, *spread, *max_spread;
  // residue form of mw_gemm: the exponents come from the leading words first; the
  // residue split sets *redo for an entry whose later word is larger (or not
  // finite, or out of range), and the pass over every word then runs again
  // (kernels that read *gate == 0 return at once).  nullptr: one pass.
  int32_t *redo;
  const int32_t *gate;
};
int launch_split(const SplitArgs &a, bool exponents_only, cudaStream_t s);

// ---- plain FP64 form (mw_plain.cu) -------------------------------------------
struct PlainArgs {
  int m, w, S_A, S_B, D;
  int64_t M, N, Kp;            // Kp: padded reduction length (digit row stride)
  const double *dA, *dB;        // S_A x M x Kp, S_B x N x Kp pieces
  const int32_t *eA, *eB;       // row / column exponents
  double *C;
  int64_t ldc, psc;
};
int launch_plain(const PlainArgs &a, cudaStream_t s);

// ---- Ozaki form (mw_ozaki.cu) ------------------------------------------------
struct OzakiArgs {
  int m, w, S_A, S_B, D, group, chunk;
  bool crt;                     // residue form: S_A, S_B fixed-point bits, D moduli
  int64_t M, N, Kp;
  const void *dA, *dB;          // bf16 pieces, S x rows x Kp
  const int32_t *eA, *eB;
  void *partials;               // partial sums (see narrow_partials), then the work counter
  double *C;
  int64_t ldc, psc;
};
// The product kernel for one problem (info == nullptr: M, N, K) or a batch
// (info, hdr: device arrays written by the batched prologue, mw_work.cuh).
// Pieces per entry the inner-product kernel is compiled for (w = 24).
int dot_pieces_range(int m, int *lo, int *hi);

// Profiling hook of mw_set_phase_events: records event i on s while set.
void phase(int i, cudaStream_t s);

struct ProductLaunch {
  const void *pieceA, *pieceB;  // bf16 pieces, rows of Kpitch (A) and KpitchB (B) elements
  int64_t rowsA, rowsB, Kpitch, KpitchB;
  int S_A, S_B, D, w, group, chunk;
  const void *info, *hdr;
  const int32_t *item_problem;    // batches: problem of every work item, or nullptr
  int count;
  int64_t M, N, K;
  void *partials;                 // int32 [t][M][N] (narrow) or int64 [g][M][N]
  bool narrow;
  bool crt;                       // residue form: one product per modulus t < D
  unsigned long long *next_item;  // work counter (reset by launch_product)
};
int launch_product(const ProductLaunch &a, cudaStream_t s);

// Exact fusion and rounding of one product's partial sums (mw_combine.cu).
int launch_combine(const OzakiArgs &a, int G, bool narrow, cudaStream_t s);
// between_kernels runs after the product kernel is launched, before the combine.
int launch_ozaki(const OzakiArgs &a, cudaStream_t s, const std::function<void()> &between_kernels);
// Every diagonal sum s_t fits in int32: S_min * K * 2^(2w-2) < 2^31.  Then the
// partial sums are the int32 s_t, otherwise int64 group sums; every plane is
// column-major (entry (i, j) at j M + i).
bool narrow_partials(int S_A, int S_B, int w, int64_t max_K);
size_t ozaki_partials_planes_bytes(int64_t M, int64_t N, int D, int group, bool narrow);
size_t ozaki_partials_bytes(int64_t M, int64_t N, int D, int group, bool narrow);
// Residue form: the product kernel stores the balanced residue of every sum as
// bfloat16 in row-major planes: entry (i, j) of modulus t at (t M + i) crt_ld(N)
// + j, crt_ld(N) a multiple of 8 (rows start on 16-byte boundaries and
// tensor-map strides are multiples of 16 bytes).  Then the 8-byte work counter.
__host__ __device__ inline int64_t crt_ld(int64_t N) { return (N + 7) & ~(int64_t)7; }

// CTAs of `threads` threads using `regs` registers a thread that the register
// file of one SM holds: registers are given to warps in blocks of 256, and each
// of the four sub-partitions (16384 registers) holds its share of a CTA's warps.
inline int ctas_by_registers(int regs, int threads) {
  const int per_warp = ((regs < 1 ? 1 : regs) * 32 + 255) / 256 * 256;
  const int warps_per_part = 16384 / per_warp;
  const int cta_warps_per_part = ((threads + 31) / 32 + 3) / 4;
  return warps_per_part / cta_warps_per_part;
}
size_t crt_residue_planes_bytes(int64_t M, int64_t N, int D);
size_t crt_partials_bytes(int64_t M, int64_t N, int D);
// Tensor map of `rank` dimensions over a bfloat16 array (dims innermost first,
// strides in bytes of dimensions 1.., box in elements), 128-byte swizzle or
// none, zeros outside the array.  map points to a CUtensorMap (64-byte aligned).
int make_map_bf16(void *map, const void *base, int rank, const uint64_t *dims,
                  const uint64_t *strides, const uint32_t *box, bool swizzle128 = true);

// ---- textbook form (mw_textbook.cu) ---------------------------------------------
int launch_textbook(int m, int transA, int transB, int64_t M, int64_t N, int64_t K,
                    const double *A, int64_t lda, int64_t psa, const double *B, int64_t ldb,
                    int64_t psb, double *C, int64_t ldc, int64_t psc, cudaStream_t s);
int launch_elementwise(int op, int m, int64_t n, const double *A, int64_t psa, const double *B,
                       int64_t psb, double *C, int64_t psc, cudaStream_t s);

// ---- residue form (mw_crt.cu) -------------------------------------------------
constexpr int kCrtMaxModuli = 96;   // capacity of the moduli tables
constexpr int kCrtMaxLimbs = 24;    // 32-bit limbs of the largest modulus product
int crt_table_size();               // moduli in the library's table
int crt_modulus(int i);             // modulus i of the table (0 past its end)
int crt_chunk(int i);               // products per fp32 accumulation: 256, 128 or 64
double crt_bits(int n);             // log2 of the product of the first n moduli
// Balanced residues of the fixed-point values (a.S bits) modulo the first
// a.nmod moduli, bfloat16 planes laid out as mw_split's digits.
int launch_residues(const SplitArgs &a, cudaStream_t s);
// Reconstruction of the exact products from the D int32 planes of the product
// kernel and greedy rounding into m words.
int launch_crt_combine(const OzakiArgs &a, cudaStream_t s);

// Number of diagonal groups.
inline int n_groups(int D, int group) { return (D + group - 1) / group; }

// Diagonals per work item of the product kernel.  Narrow partial sums are per
// diagonal, so a work item can be a single diagonal (fine-grained load
// balance, at most 64 items per tile); wide ones need the plan's int64 group.
inline int sched_group(int D, int group, bool narrow) {
  return narrow ? (D + 63) / 64 : group;
}

}  // namespace mw
