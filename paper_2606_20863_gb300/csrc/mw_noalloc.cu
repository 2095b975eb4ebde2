// mw_gemm_noalloc: the Ozaki / plain product for callers that cannot allocate
// device memory.
//
// mw_gemm needs a workspace (exponents, pieces, partial sums) that the caller
// allocates.  Some callers cannot do that: a plug-in living inside a host
// program that owns every byte of device memory through its own pool (a
// framework's caching allocator, a server with a fixed memory budget) may not
// call cudaMalloc, which synchronizes the device and takes memory the host
// does not account for, and code that must not fail half-way for lack of
// memory wants its storage reserved before it runs.  This entry point takes
// its workspace from a fixed array that the library reserves on every device
// it is loaded on and keeps until the process exits.
//
// The array is shared by every call on a device and keeps what the last call
// left in it; mw_gemm clears the few words it needs zeroed (the exponent and
// spread accumulators) on every call, so nothing else has to start at zero.
// Two calls whose work overlaps on the GPU (different streams, not ordered)
// race on the array.
#include <mutex>

#include "mw_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB per device

// In host code this name is only a stand-in for the device array: its device
// address comes from cudaGetSymbolAddress with the device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the array on the current device.  Outside a stream capture
// it is looked up on every call (cheap), so that a context created anew on the
// device (after cudaDeviceReset, say), where the array may sit elsewhere, never
// gets a stale address; inside a capture the address of the last call outside
// it is used, since the first lookup may load the library's module, which a
// capture does not allow.
int scratch_of_current_device(cudaStream_t stream, void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mw::cuda_fail(e, "mw_gemm_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return mw::fail(MW_EUNSUPPORTED, "device %d out of range", dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return mw::cuda_fail(e, "mw_gemm_noalloc: cudaStreamIsCapturing");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return mw::cuda_fail(e, "mw_gemm_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  } else if (!g_scratch_addr[dev]) {
    return mw::fail(MW_EINVAL, "mw_gemm_noalloc: the first call on a device must come before "
                               "any stream capture");
  }
  *out = g_scratch_addr[dev];
  return MW_OK;
}

}  // namespace

extern "C" int mw_gemm_noalloc(const mw_plan *plan, int transA, int transB, int64_t M, int64_t N,
                               int64_t K, const double *A, int64_t lda, int64_t plane_stride_a,
                               const double *B, int64_t ldb, int64_t plane_stride_b, double *C,
                               int64_t ldc, int64_t plane_stride_c, mw_stream_t stream) {
  size_t need = 0;
  int rc = mw_gemm_workspace_size(plan, M, N, K, &need);
  if (rc) return rc;
  if (need > kScratchBytes)
    return mw::fail(MW_ENOSPC,
                    "mw_gemm_noalloc: this product needs %zu bytes of scratch, the built-in "
                    "scratch holds %zu bytes; use mw_gemm with a caller-allocated workspace",
                    need, kScratchBytes);
  void *scratch = nullptr;
  if ((rc = scratch_of_current_device((cudaStream_t)stream, &scratch))) return rc;
  return mw_gemm(plan, transA, transB, M, N, K, A, lda, plane_stride_a, B, ldb, plane_stride_b,
                 C, ldc, plane_stride_c, scratch, kScratchBytes, stream);
}
