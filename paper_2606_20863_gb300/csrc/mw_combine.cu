// Step 4 of one product in the Ozaki form (MW_OZAKI): exact fusion of the
// diagonal partial sums of the product kernel (mw_ozaki.cu) and greedy rounding
// to m words, one thread per output.
#include <cuda.h>

#include <cmath>

#include "mw_column.cuh"
#include "mw_device.cuh"
#include "mw_fuse.cuh"
#include "mw_internal.h"

namespace mw {
namespace {

// ---- fusion of one product: thread per output ---------------------------------
// Narrow: D planes of int32 diagonal sums s_t, weight 2^(w (D-1-t)).
// Wide:   G planes of int64 group sums, weight 2^(w (D-1-t1_g)).
// Planes are column-major (entry (i, j) at j M + i): threads run along i.
template <int MW, int NL, bool NARROW>
__global__ void combine_kernel(const void *__restrict__ partials, const int32_t *eA,
                               const int32_t *eB, int64_t M, int64_t N, int G, int group, int D,
                               int w, double *C, int64_t ldc, int64_t psc) {
  __shared__ uint32_t limbs[2 * NL][128];          // this thread's column: limbs[*][threadIdx.x]
  const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x, j = blockIdx.y;
  if (i >= M || j >= N) return;
  uint32_t U[2 * NL];
  if (NARROW && w == 8) {
    fuse_w8<2 * NL>(U, static_cast<const int32_t *>(partials) + j * M + i, N * M, D);
  } else {
    uint64_t X[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) X[k] = 0;
    if constexpr (NARROW) {
      fuse_diagonals<NL>(X, static_cast<const int32_t *>(partials) + j * M + i, N * M, D, group, w);
    } else {
      const int64_t *p = static_cast<const int64_t *>(partials);
      for (int g = 0; g < G; ++g) {
        const int t1 = min(D, (g + 1) * group) - 1;
        add_shifted<NL>(X, p[((int64_t)g * N + j) * M + i], w * (D - 1 - t1));
      }
    }
    to_limbs32<NL>(X, U);
  }
  double *c = C + i * ldc + j;
  round_column<MW, 2 * NL>(U, &limbs[0][threadIdx.x], 128, eA[i] + eB[j] + 4 - w * (D + 1),
                           [&](int k, double v) { c[k * psc] = v; });
}

template <int MW, int NL>
int launch_combine_t(const OzakiArgs &a, int G, bool narrow, cudaStream_t s) {
  dim3 grid((unsigned)((a.M + 127) / 128), (unsigned)a.N);
  if (narrow)
    combine_kernel<MW, NL, true><<<grid, 128, 0, s>>>(a.partials, a.eA, a.eB, a.M, a.N, G, a.group,
                                                      a.D, a.w, a.C, a.ldc, a.psc);
  else
    combine_kernel<MW, NL, false><<<grid, 128, 0, s>>>(a.partials, a.eA, a.eB, a.M, a.N, G,
                                                       a.group, a.D, a.w, a.C, a.ldc, a.psc);
  return cuda_fail(cudaGetLastError(), "combine launch");
}

template <int MW>
int launch_combine_nl(const OzakiArgs &a, int G, bool narrow, cudaStream_t s) {
  // |X| < 2^(63 + w (D-1)) plus a sign bit; as few 64-bit limbs as hold it (the
  // fusion touches every limb)
  const int bits = 64 + a.w * (a.D - 1) + 1;
  if constexpr (MW == 16) {
    if (bits <= 768) return launch_combine_t<MW, 12>(a, G, narrow, s);
    if (bits <= 832) return launch_combine_t<MW, 13>(a, G, narrow, s);
    if (bits <= 896) return launch_combine_t<MW, 14>(a, G, narrow, s);
    if (bits <= 960) return launch_combine_t<MW, 15>(a, G, narrow, s);
    if (bits <= 1024) return launch_combine_t<MW, 16>(a, G, narrow, s);
    if (bits <= 1088) return launch_combine_t<MW, 17>(a, G, narrow, s);
  } else {
    if (bits <= 256) return launch_combine_t<MW, 4>(a, G, narrow, s);
    if (bits <= 320) return launch_combine_t<MW, 5>(a, G, narrow, s);
    if (bits <= 384) return launch_combine_t<MW, 6>(a, G, narrow, s);
    if (bits <= 448) return launch_combine_t<MW, 7>(a, G, narrow, s);
    if (bits <= 512) return launch_combine_t<MW, 8>(a, G, narrow, s);
    if (bits <= 576) return launch_combine_t<MW, 9>(a, G, narrow, s);
    if (bits <= 640) return launch_combine_t<MW, 10>(a, G, narrow, s);
  }
  return fail(MW_EUNSUPPORTED, "D = %d diagonals of %d bits too many for the fusion", a.D, a.w);
}

}  // namespace

int launch_combine(const OzakiArgs &a, int G, bool narrow, cudaStream_t s) {
  switch (a.m) {
    case 2: return launch_combine_nl<2>(a, G, narrow, s);
    case 4: return launch_combine_nl<4>(a, G, narrow, s);
    case 8: return launch_combine_nl<8>(a, G, narrow, s);
    case 16: return launch_combine_nl<16>(a, G, narrow, s);
  }
  return fail(MW_EINVAL, "m must be 2, 4, 8 or 16");
}

}  // namespace mw
