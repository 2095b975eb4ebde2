// Description of the products a product kernel works on (device side, shared
// by the single and batched paths).  A work item is (problem, diagonal group,
// output tile); items are numbered problem by problem.
#pragma once
#include <cstdint>

namespace mw {
namespace {

struct BInfo {            // one problem, filled by the prologue
  int64_t M, N, K;
  const double *A;
  int64_t lda, psa;
  const double *B;
  int64_t ldb, psb;
  double *C;
  int64_t ldc, psc;
  int64_t rowA, rowB;     // first piece row of the problem in the A / B piece arrays
  int64_t eA, eB;         // prefix sums of M and N: exponent offsets
  int64_t part;           // offset of the partial sums (int64 units)
  int64_t work;           // first work item
  int64_t outs;           // prefix sum of M*N: first output in the flat output order
  int64_t stripes;        // prefix sum of ceil(N/32): first 32-column stripe of B
  int32_t tiles_m, tiles_n, KB;
  // rs: B slices side by side in one MMA (column block j of the accumulator is
  // diagonal t + j); the piece rows of B then hold rs - 1 zero slices before
  // slice 0 and after slice S_B - 1, slice q at rowB + (q + rs - 1) N.
  // nd: diagonals per work item; G: work items per output tile.
  int32_t rs, nd, G;
  // K-packed pieces (narrow batches): K8 = K rounded up to 8; a row of A holds its
  // slices back to back (slice p at column p K8), a row of B (a column of B_i)
  // its slices in descending order after Z K8 zero columns (slice q at column
  // (Z + S_B - 1 - q) K8) and (rs - 1) K8 + 64 zeros, rounded up to K8, after
  // them; Z = rs - 1 (the reads of stacked block j start j K8 lower).
  int32_t K8, Z;
};

struct BHeader {          // written by the prologue
  int64_t sum_M, sum_N, sum_MN, total_work;
  int32_t bad;            // the descriptors disagree with the host summary
  int32_t max_spread[2];
  int32_t pad;
  unsigned long long next_item;  // work counter of the product kernel
  int64_t sum_stripes;           // 32-column stripes of all B_i
};

// problem owning flat index x, given a field that holds exclusive prefix sums
template <typename F>
__device__ __forceinline__ int find_problem(const BInfo *info, int count, int64_t x, F key) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (key(info[mid]) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace
}  // namespace mw
