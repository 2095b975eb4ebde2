// MW_OZAKI: step 3 of the error-free summation on the tcgen05 tensor cores,
// step 4 as exact integer fusion.
//
// Section 4 observes that the diagonal convolutions s_i turn an m-double inner
// product into matrix products of pieces, "in particular tensor cores", the
// Ozaki scheme of Section 1.  Pieces are balanced integers |d| <= 2^(w-1),
// w in {7, 8}, stored in bfloat16 (exact); a product of two pieces is at most
// 2^(2w-2) and a sum of `chunk` of them is at most 2^22, so the fp32
// accumulators of the tensor core hold exact integers.  After every chunk the
// accumulator is drained from tensor memory into 64-bit integers:
//   v + 1.5*2^23 (one fp32 add, exact for |v| <= 2^22) has bit pattern
//   0x4B400000 + v, which is added as an unsigned 32-bit value; the constant
//   is subtracted once per group (arithmetic mod 2^64, exact because the true
//   group value fits in int64).
// A group of `group` consecutive diagonals t0..t1 is fused by Horner's rule,
// V = sum_t s_t 2^(w (t1 - t)), and written to the partial-sum buffer; the
// combine kernel adds the groups exactly, X = sum_g V_g 2^(w (D-1-t1_g)), and
// rounds X 2^(E_i + E_j + 4 - w(D+1)) to nearest into m words, one after the
// other (greedy), all in integer arithmetic.
//
// Kernel layout (one 128 x 128 output tile per work unit, one CTA per SM):
//   warp 0      TMA producer: piece tiles 128 x 64 of A_p and B_q per stage
//   warp 1      tensor-memory allocation and the single MMA-issuing thread
//   warps 2..9  drain: warp w reads TMEM lanes 32 (w % 4).., columns 64 ((w-2)/4)..
// A work unit is (diagonal group, output tile); units are spread over
// persistent CTAs.  Every wait is bounded (mbar_wait).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "mw_device.cuh"

namespace mw {
namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int STAGES = 6;
constexpr int NUM_DRAIN_WARPS = 8;
constexpr int NUM_THREADS = 64 + 32 * NUM_DRAIN_WARPS;
constexpr int TMEM_COLS = 2 * BN;
constexpr uint32_t STAGE_A = BM * BK * 2, STAGE_B = BN * BK * 2;
constexpr uint32_t MAGIC_BITS = 0x4B400000u;  // bit pattern of 1.5 * 2^23
constexpr int MAX_GROUPS = 64;
constexpr size_t SMEM_BYTES = 1024 + STAGES * (STAGE_A + STAGE_B) + 256;

struct Params {
  int KB;                 // k-blocks of 64 per piece row
  int S_A, S_B, D, w, group, G, chunk_kb;
  int tiles_m, tiles_n, units;
  int64_t *partials;
  unsigned int *status;
  int gorder[MAX_GROUPS]; // groups, most expensive first
};

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// 32 lanes x 32 columns of 32-bit words; thread i gets lane (base + i), 32 columns.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the layout a 128-byte-swizzled TMA box of 64 bf16 wide
// leaves behind).  Fields: start address >> 4 (bits 0-13), leading byte offset
// >> 4 (16-29, unused for this layout), stride byte offset >> 4 (32-45),
// descriptor version 1 (46-47), swizzle mode 2 = 128 B (61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: fp32 accumulator (bits 4-5 = 1), A and B
// bfloat16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

struct Unit {
  int g, t0, t1, tm, tn, tile;
};
__device__ __forceinline__ Unit decode(const Params &P, int u) {
  const int tiles = P.tiles_m * P.tiles_n;
  Unit x;
  x.g = P.gorder[u / tiles];
  x.tile = u % tiles;
  x.tm = x.tile % P.tiles_m;
  x.tn = x.tile / P.tiles_m;
  x.t0 = x.g * P.group;
  x.t1 = min(P.D, x.t0 + P.group) - 1;
  return x;
}
__device__ __forceinline__ int plo(const Params &P, int t) { return max(0, t - P.S_B + 1); }
__device__ __forceinline__ int phi(const Params &P, int t) { return min(t, P.S_A - 1); }
__device__ __forceinline__ int nsteps(const Params &P, int t) {
  const int n = phi(P, t) - plo(P, t) + 1;
  return n > 0 ? n * P.KB : 0;
}
__device__ __forceinline__ int nchunks(const Params &P, int t) {
  return (nsteps(P, t) + P.chunk_kb - 1) / P.chunk_kb;
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    ozaki_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                 const Params P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * STAGE_A;
  uint64_t *full = (uint64_t *)(smem + STAGES * (STAGE_A + STAGE_B));
  uint64_t *empty = full + STAGES;
  uint64_t *accf = empty + STAGES;
  uint64_t *acce = accf + 2;
  uint64_t *done = acce + 2;
  uint32_t *tmem_holder = (uint32_t *)(done + 1);
  volatile int *abort = (volatile int *)(tmem_holder + 1);
  int *counters = (int *)(tmem_holder + 2);  // [0] TMA steps issued, [1] consumed

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], NUM_DRAIN_WARPS);
    }
    mbar_init(done, 1);
    *abort = 0;
    counters[0] = counters[1] = 0;
    fence_barrier_init();
    prefetch_map(&mapA);
    prefetch_map(&mapB);
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
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      uint32_t it = 0;
      for (int u = blockIdx.x; u < P.units && !*abort; u += gridDim.x) {
        const Unit x = decode(P, u);
        for (int t = x.t0; t <= x.t1 && !*abort; ++t) {
          for (int p = plo(P, t); p <= phi(P, t) && !*abort; ++p) {
            const int q = t - p;
            for (int kb = 0; kb < P.KB; ++kb, ++it) {
              const uint32_t s = it % STAGES, ph = (it / STAGES) & 1;
              if (!mbar_wait(&empty[s], ph ^ 1, P.status, abort)) break;
              mbar_arrive_expect_tx(&full[s], STAGE_A + STAGE_B);
              tma_load_3d(smem_u32(sA + s * STAGE_A), &mapA, kb * BK, x.tm * BM, p,
                          smem_u32(&full[s]));
              tma_load_3d(smem_u32(sB + s * STAGE_B), &mapB, kb * BK, x.tn * BN, q,
                          smem_u32(&full[s]));
              counters[0] = (int)it + 1;
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t it = 0, ch = 0;
      for (int u = blockIdx.x; u < P.units && !*abort; u += gridDim.x) {
        const Unit x = decode(P, u);
        for (int t = x.t0; t <= x.t1 && !*abort; ++t) {
          const int total = nsteps(P, t);
          for (int j = 0; j < total && !*abort; ++ch) {
            const int nk = min(P.chunk_kb, total - j);
            const uint32_t b = ch & 1, bph = (ch >> 1) & 1;
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
                tc_mma(d, ad + 2 * kk, bd + 2 * kk, kIdesc, (jj | kk) ? 1u : 0u);
              tc_commit(&empty[s]);
              counters[1] = (int)it + 1;
            }
            tc_commit(&accf[b]);
            j += nk;
          }
        }
      }
      // make sure every MMA issued has completed before teardown (this wait
      // ignores the abort flag: it only ends early on its own time limit)
      tc_commit(done);
      volatile int never = 0;
      mbar_wait(done, 0, P.status, &never);
    }
  } else {
    // ---------------- drain warps ----------------
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + half * 64;
    const int tiles = P.tiles_m * P.tiles_n;
    uint32_t ch = 0;
    uint64_t acc[64];
    bool ok = true;
    for (int u = blockIdx.x; u < P.units && ok; u += gridDim.x) {
      const Unit x = decode(P, u);
#pragma unroll
      for (int i = 0; i < 64; ++i) acc[i] = 0;
      uint64_t bias = 0;
      for (int t = x.t0; t <= x.t1 && ok; ++t) {
        if (t > x.t0) {
#pragma unroll
          for (int i = 0; i < 64; ++i) acc[i] <<= P.w;
          bias <<= P.w;
        }
        const int nch = nchunks(P, t);
        bias += (uint64_t)nch * MAGIC_BITS;
        for (int c = 0; c < nch; ++c, ++ch) {
          const uint32_t b = ch & 1, bph = (ch >> 1) & 1;
          // warp-uniform outcome: tcgen05.ld below needs every lane of the warp
          if (!__all_sync(0xffffffffu, mbar_wait(&accf[b], bph, P.status, abort))) {
            ok = false;
            break;
          }
          tc_fence_after();
          uint32_t v[32];
          tc_ld32(tbase + b * BN, v);
          tc_wait_ld();
#pragma unroll
          for (int i = 0; i < 32; ++i)
            acc[i] += __float_as_uint(__uint_as_float(v[i]) + 12582912.0f);
          tc_ld32(tbase + b * BN + 32, v);
          tc_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce[b]);
#pragma unroll
          for (int i = 0; i < 32; ++i)
            acc[32 + i] += __float_as_uint(__uint_as_float(v[i]) + 12582912.0f);
        }
      }
      if (!ok) break;
      // partial sums row-major within the tile: 64 consecutive columns per thread
      longlong2 *dst = reinterpret_cast<longlong2 *>(
          P.partials + ((size_t)(x.g * tiles + x.tile) * BM + row) * BN + half * 64);
#pragma unroll
      for (int i = 0; i < 32; ++i)
        dst[i] = make_longlong2((long long)(acc[2 * i] - bias), (long long)(acc[2 * i + 1] - bias));
    }
  }

  __syncthreads();
  if (warp == 0 && lane == 0 && *abort) {
    // let the copies still in flight land before the shared memory goes away
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

// ---- combine: exact fusion of the group partial sums -------------------------
template <int NL>
__device__ __forceinline__ bool is_zero(const uint64_t (&x)[NL]) {
  uint64_t o = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i) o |= x[i];
  return o == 0;
}

// Shift left so that bit 63 of the top limb is set; returns the shift.
template <int NL>
__device__ __forceinline__ int normalize(uint64_t (&x)[NL]) {
  int sh = 0;
  // whole limbs first
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    if (x[NL - 1] == 0) {
#pragma unroll
      for (int i = NL - 1; i > 0; --i) x[i] = x[i - 1];
      x[0] = 0;
      sh += 64;
    }
  }
  const int b = __clzll((long long)x[NL - 1]);
  if (b) {
#pragma unroll
    for (int i = NL - 1; i > 0; --i) x[i] = (x[i] << b) | (x[i - 1] >> (64 - b));
    x[0] <<= b;
  }
  return sh + b;
}

template <int MW, int NL>
__global__ void combine_kernel(const int64_t *__restrict__ partials, const int32_t *eA,
                               const int32_t *eB, int64_t M, int64_t N, int tiles_m, int tiles_n,
                               int G, int group, int D, int w, double *C, int64_t ldc,
                               int64_t psc) {
  const int tiles = tiles_m * tiles_n;
  {
    const int64_t j = (int64_t)blockIdx.x * 128 + threadIdx.x, i = blockIdx.y;
    double words[MW];
#pragma unroll
    for (int k = 0; k < MW; ++k) words[k] = 0.0;
    if (i < M && j < N) {
      const int tile = (int)(j / BN) * tiles_m + (int)(i / BM);
      const int64_t off = (int64_t)(i % BM) * BN + (j % BN);
      // X = sum_g V_g 2^(w (D - 1 - t1_g)), two's complement in NL limbs
      uint64_t X[NL];
#pragma unroll
      for (int k = 0; k < NL; ++k) X[k] = 0;
      for (int g = 0; g < G; ++g) {
        const int64_t V = partials[(size_t)(g * tiles + tile) * BN * BM + off];
        const int t1 = min(D, (g + 1) * group) - 1;
        const int sh = w * (D - 1 - t1);
        const int li = sh >> 6, bo = sh & 63;
        const uint64_t lo = (uint64_t)V << bo;
        const uint64_t hi = bo ? (uint64_t)(V >> (64 - bo)) : (uint64_t)(V >> 63);
        const uint64_t ext = (uint64_t)(V >> 63);
        uint64_t carry = 0;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
          const uint64_t a = k < li ? 0 : (k == li ? lo : (k == li + 1 ? hi : ext));
          const uint64_t s1 = X[k] + a;
          const uint64_t c1 = s1 < a;
          const uint64_t s2 = s1 + carry;
          const uint64_t c2 = s2 < carry;
          X[k] = s2;
          carry = c1 | c2;
        }
      }
      // magnitude and sign
      bool neg = (int64_t)X[NL - 1] < 0;
      if (neg) {
        uint64_t c = 1;
#pragma unroll
        for (int k = 0; k < NL; ++k) {
          const uint64_t s = ~X[k] + c;
          c = (s == 0 && c) ? 1 : 0;
          X[k] = s;
        }
      }
      // value = X 2^ex; greedy rounding to nearest, ties to even, word by word
      int ex = eA[i] + eB[j] + 4 - w * (D + 1);
#pragma unroll
      for (int k = 0; k < MW; ++k) {
        if (is_zero<NL>(X)) break;
        ex -= normalize<NL>(X);
        const uint64_t top = X[NL - 1];
        uint64_t mant = top >> 11;
        const uint64_t rbit = (top >> 10) & 1;
        uint64_t sticky = top & 0x3FF;
#pragma unroll
        for (int q = 0; q < NL - 1; ++q) sticky |= X[q];
        const uint64_t up = rbit & ((sticky != 0) | (mant & 1));
        mant += up;
        const double mag = scalbn((double)mant, ex + 64 * (NL - 1) + 11);
        words[k] = neg ? -mag : mag;
        // remainder: low bits minus (up ? 2^pos : 0), pos = 64 (NL-1) + 11
        X[NL - 1] = top & 0x7FF;
        if (up) {
          // X <- 2^pos - low, sign flips
          X[NL - 1] = (~X[NL - 1]) & 0x7FF;
#pragma unroll
          for (int q = 0; q < NL - 1; ++q) X[q] = ~X[q];
          uint64_t c = 1;
#pragma unroll
          for (int q = 0; q < NL; ++q) {
            const uint64_t s = X[q] + c;
            c = (s == 0 && c) ? 1 : 0;
            X[q] = s;
          }
          neg = !neg;
        }
      }
    }
    if (i < M && j < N)
#pragma unroll
      for (int k = 0; k < MW; ++k) C[k * psc + i * ldc + j] = words[k];
  }
}

template <int MW, int NL>
int launch_combine(const OzakiArgs &a, int tiles_m, int tiles_n, int G, cudaStream_t s) {
  dim3 grid((unsigned)((a.N + 127) / 128), (unsigned)a.M);
  combine_kernel<MW, NL><<<grid, 128, 0, s>>>(a.partials, a.eA, a.eB, a.M, a.N, tiles_m,
                                                       tiles_n, G, a.group, a.D, a.w, a.C, a.ldc,
                                                       a.psc);
  return cuda_fail(cudaGetLastError(), "combine launch");
}

template <int MW>
int launch_combine_nl(const OzakiArgs &a, int tiles_m, int tiles_n, int G, cudaStream_t s) {
  // |X| < 2^(63 + w (D-1)) plus a sign bit
  const int bits = 64 + a.w * (a.D - 1) + 1;
  if (bits <= 256) return launch_combine<MW, 4>(a, tiles_m, tiles_n, G, s);
  if (bits <= 384) return launch_combine<MW, 6>(a, tiles_m, tiles_n, G, s);
  if (bits <= 512) return launch_combine<MW, 8>(a, tiles_m, tiles_n, G, s);
  if (bits <= 640) return launch_combine<MW, 10>(a, tiles_m, tiles_n, G, s);
  return fail(MW_EUNSUPPORTED, "D = %d diagonals of %d bits too many for the combine", a.D, a.w);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

int make_map(CUtensorMap *map, const void *base, int64_t Kp, int64_t rows, int S, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fail(MW_ECUDA, "cuTensorMapEncodeTiled not available");
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)(Kp * rows * 2)};
  cuuint32_t box[3] = {BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(MW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return MW_OK;
}

}  // namespace

size_t ozaki_partials_bytes(int64_t M, int64_t N, int D, int group) {
  const int64_t tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  return (size_t)n_groups(D, group) * tm * tn * BM * BN * sizeof(int64_t);
}

int launch_ozaki(const OzakiArgs &a, cudaStream_t s, const std::function<void()> &between_kernels) {
  if (a.Kp % BK) return fail(MW_EINVAL, "padded K must be a multiple of %d", BK);
  if (a.chunk < BK || a.chunk % BK) return fail(MW_EINVAL, "chunk must be a positive multiple of 64");
  if (a.w < 2 || a.w > 8 || (int64_t)a.chunk << (2 * a.w - 2) > (1 << 22))
    return fail(MW_EINVAL, "chunk * 2^(2w-2) must not exceed 2^22 (w=%d chunk=%d)", a.w, a.chunk);
  const int G = n_groups(a.D, a.group);
  if (G > MAX_GROUPS) return fail(MW_EUNSUPPORTED, "more than %d diagonal groups", MAX_GROUPS);
  Params P{};
  P.KB = (int)(a.Kp / BK);
  P.S_A = a.S_A;
  P.S_B = a.S_B;
  P.D = a.D;
  P.w = a.w;
  P.group = a.group;
  P.G = G;
  P.chunk_kb = a.chunk / BK;
  P.tiles_m = (int)((a.M + BM - 1) / BM);
  P.tiles_n = (int)((a.N + BN - 1) / BN);
  P.units = G * P.tiles_m * P.tiles_n;
  P.partials = a.partials;
  P.status = status_ptr();
  // most expensive groups first (pairs per diagonal grow, then shrink)
  long long cost[MAX_GROUPS];
  for (int g = 0; g < G; ++g) {
    cost[g] = 0;
    for (int t = g * a.group; t < std::min(a.D, (g + 1) * a.group); ++t)
      cost[g] += std::max(0, std::min(t, a.S_A - 1) - std::max(0, t - a.S_B + 1) + 1);
    P.gorder[g] = g;
  }
  for (int i = 1; i < G; ++i)
    for (int j = i; j > 0 && cost[P.gorder[j]] > cost[P.gorder[j - 1]]; --j)
      std::swap(P.gorder[j], P.gorder[j - 1]);

  CUtensorMap mA, mB;
  int rc = make_map(&mA, a.dA, a.Kp, a.M, a.S_A, BM);
  if (rc) return rc;
  if ((rc = make_map(&mB, a.dB, a.Kp, a.N, a.S_B, BN))) return rc;

  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(ozaki_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return cuda_fail(e, "ozaki smem attribute");
    attr_set = true;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::min(P.units, nsm);
  ozaki_kernel<<<grid, NUM_THREADS, SMEM_BYTES, s>>>(mA, mB, P);
  if ((rc = cuda_fail(cudaGetLastError(), "ozaki kernel launch"))) return rc;
  if (between_kernels) between_kernels();
  switch (a.m) {
    case 2: return launch_combine_nl<2>(a, P.tiles_m, P.tiles_n, G, s);
    case 4: return launch_combine_nl<4>(a, P.tiles_m, P.tiles_n, G, s);
    case 8: return launch_combine_nl<8>(a, P.tiles_m, P.tiles_n, G, s);
  }
  return fail(MW_EINVAL, "m must be 2, 4 or 8");
}

}  // namespace mw
