// Device helpers shared by the kernels of libmw (GPU side only).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mw_internal.h"

namespace mw {

// ---------------------------------------------------------------------------
// Status word: kernels OR error bits into a per-device word (mw_get_status).
__device__ __forceinline__ void raise_status(unsigned int *status, unsigned int bits) {
  if (status) atomicOr(status, bits);
}

// ---------------------------------------------------------------------------
// Exponents from the bit pattern (no floating-point unit involved).
// ilogb(x) + 1 for a nonzero finite double; kExpZero for +-0.
constexpr int kExpZero = -100000;
constexpr int kExpNonFinite = 100000;

__device__ __forceinline__ int exp_plus1(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7ff);
  const uint64_t f = b & ((1ull << 52) - 1);
  if (be == 0x7ff) return kExpNonFinite;
  if (be == 0) return f ? (63 - __clzll((long long)f)) - 1074 + 1 : kExpZero;
  return be - 1023 + 1;
}

// |x| = M 2^(e2) with M an integer < 2^53 (M = 0 for zero); returns M, sets e2, neg.
__device__ __forceinline__ uint64_t mantissa_of(double x, int &e2, bool &neg) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7ff);
  const uint64_t f = b & ((1ull << 52) - 1);
  neg = (b >> 63) != 0;
  if (be == 0) { e2 = -1074; return f; }
  e2 = be - 1075;
  return f | (1ull << 52);
}

// ---------------------------------------------------------------------------
// Bounded waits.  Every spin in the library gives up after kWaitLimitNs of
// global time, raises MW_ETIMEOUT and reports failure to the caller, which
// then stops issuing work and unwinds.
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait until the phase of `bar` with parity `parity` has completed.  Returns
// false (after raising MW_ETIMEOUT) if that takes longer than limit_ns or if
// *abort became nonzero meanwhile.
__device__ __forceinline__ bool mbar_wait_for(uint64_t *bar, uint32_t parity,
                                              unsigned int *status, volatile int *abort,
                                              uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t spin = 1;; ++spin) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spin & 255u) == 0) {
      if (*abort) return false;
      if (global_ns() - t0 > limit_ns) {
        raise_status(status, MW_ETIMEOUT);
        *abort = 1;
        return false;
      }
    }
  }
}

// The pipeline kernels' wait: limit kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned int *status,
                                          volatile int *abort) {
  return mbar_wait_for(bar, parity, status, abort, kWaitLimitNs);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile(
      "{\n .reg .b32 rx;\n .reg .pred px;\n"
      " elect.sync rx|px, 0xffffffff;\n"
      " selp.u32 %0, 1, 0, px;\n}\n"
      : "=r"(pred));
  return pred != 0;
}

}  // namespace mw
