// The C interface of libmw (include/mw.h): argument checks, the planner, the
// workspace layout, the per-device status word, and the order of launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "mw_device.cuh"
#include "mw_internal.h"

namespace mw {

namespace {
thread_local std::string g_msg;
__device__ unsigned int g_status_word;  // MW_* bits raised by kernels of this device
constexpr int kMaxDevices = 64;
unsigned int *g_status_addr[kMaxDevices] = {nullptr};
std::mutex g_status_mu;
cudaEvent_t g_phase[4] = {nullptr, nullptr, nullptr, nullptr};
bool g_phase_on = false;

}  // namespace

void phase(int i, cudaStream_t s) {
  if (g_phase_on && g_phase[i]) cudaEventRecord(g_phase[i], s);
}

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_msg = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return MW_OK;
  return fail(MW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Device address of g_status_word on the current device.  In host code the
// symbol's name is only a stand-in, so the address is looked up once per
// device with that device current.
unsigned int *status_ptr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_status_mu);
  if (!g_status_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
    g_status_addr[dev] = static_cast<unsigned int *>(p);
  }
  return g_status_addr[dev];
}

namespace {

// m = 16 (hexa doubles) runs the tensor-core form and inner products only
bool valid_m(int m) { return m == 2 || m == 4 || m == 8 || m == 16; }

int ceil_div_bits(double bits, int w) {
  const int n = (int)std::ceil(bits / w - 1e-9);
  return n < 1 ? 1 : n;
}

// Largest group g of consecutive diagonals whose Horner sum fits in int64.
int group_size(int S_min, int64_t K, int w) {
  const int bits_s = (int)std::ceil(std::log2((double)S_min * (double)K)) + 2 * w - 2;
  if (bits_s > 62) return 0;
  return (62 - bits_s) / w + 1;
}

struct Layout {
  size_t exps, digA, digB, partials, total;
  int64_t Kp;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(const mw_plan &p, int64_t M, int64_t N, int64_t K) {
  Layout L{};
  L.Kp = round_up(K, 64);
  if (p.mode == MW_TEXTBOOK) {       // no pieces, no partial sums
    L.total = 256;
    return L;
  }
  const size_t elem = p.mode == MW_PLAIN ? 8 : 2;
  // planes of pieces: S_A / S_B digits, or D residues in the residue form
  const size_t planesA = p.mode == MW_CRT ? p.D : p.S_A, planesB = p.mode == MW_CRT ? p.D : p.S_B;
  L.exps = 0;
  // exponents and spreads of both operands, the largest spreads, the redo flags
  size_t off = align256(sizeof(int32_t) * (2 * (size_t)M + 2 * (size_t)N + 4));
  L.digA = off;
  off = align256(off + planesA * M * L.Kp * elem);
  L.digB = off;
  off = align256(off + planesB * N * L.Kp * elem);
  L.partials = off;
  if (p.mode == MW_OZAKI)
    off = align256(off + ozaki_partials_bytes(M, N, p.D, p.group,
                                              narrow_partials(p.S_A, p.S_B, p.w, L.Kp)));
  else if (p.mode == MW_CRT)
    off = align256(off + crt_partials_bytes(M, N, p.D));
  L.total = off;
  return L;
}

int check_plan(const mw_plan *p, int64_t M, int64_t N, int64_t K) {
  if (!p) return fail(MW_EINVAL, "plan is NULL");
  if (!valid_m(p->m)) return fail(MW_EINVAL, "m = %d, must be 2, 4, 8 or 16", p->m);
  if (M <= 0 || N <= 0 || K <= 0) return fail(MW_EINVAL, "dimensions must be positive");
  if (p->mode != MW_TEXTBOOK && (p->S_A < 1 || p->S_B < 1 || p->D < 1))
    return fail(MW_EINVAL, "S_A, S_B, D must be >= 1");
  if (p->mode == MW_OZAKI) {
    if (p->w < 2 || p->w > 8) return fail(MW_EINVAL, "Ozaki piece width w must be 2..8");
    if (p->group < 1 || p->chunk < 64) return fail(MW_EINVAL, "bad group/chunk");
    const int S_min = p->S_A < p->S_B ? p->S_A : p->S_B;
    const int gmax = group_size(S_min, K, p->w);
    if (gmax < 1 || p->group > gmax)
      return fail(MW_EINVAL, "group %d exceeds the int64 limit %d", p->group, gmax);
  } else if (p->mode == MW_TEXTBOOK) {
    if (p->m != 2 && p->m != 4 && p->m != 8)
      return fail(MW_EUNSUPPORTED, "the textbook form (MW_TEXTBOOK) takes m = 2, 4 and 8");
  } else if (p->mode == MW_CRT) {
    if (p->m != 2 && p->m != 4)
      return fail(MW_EUNSUPPORTED, "the residue form (MW_CRT) takes m = 2 and 4");
    if (p->w != 1) return fail(MW_EINVAL, "MW_CRT plans have w = 1 (S_A, S_B are bits)");
    if (p->S_A < 2 || p->S_B < 2 || p->S_A > 381 || p->S_B > 381)
      return fail(MW_EUNSUPPORTED, "MW_CRT fixed-point bits must be 2..381");
    if (p->D > crt_table_size())
      return fail(MW_EUNSUPPORTED, "MW_CRT: %d moduli, the table has %d", p->D, crt_table_size());
    const double need = p->S_A + p->S_B + 1 + std::log2((double)K);
    if (crt_bits(p->D) <= need)
      return fail(MW_EINVAL, "MW_CRT: %d moduli hold %.1f bits, the products need %.1f", p->D,
                  crt_bits(p->D), need);
  } else if (p->mode == MW_PLAIN) {
    if (p->m == 16) return fail(MW_EUNSUPPORTED, "m = 16 has no MW_PLAIN form (MW_OZAKI and MW_DOT take it)");
    if (p->w < 1 || p->w > 26) return fail(MW_EINVAL, "plain piece width w must be 1..26");
    const int S_min = p->S_A < p->S_B ? p->S_A : p->S_B;
    const double bits = std::log2((double)S_min * (double)K) + 2.0 * p->w - 2.0;
    if (bits > 53.0) return fail(MW_EINVAL, "plain plan not exact: pairs*K*2^(2w-2) > 2^53");
  } else {
    return fail(MW_EINVAL, "mode must be MW_PLAIN, MW_OZAKI, MW_CRT or MW_TEXTBOOK");
  }
  return MW_OK;
}

int check_mat(const double *X, int64_t rows, int64_t cols, int64_t ld, int64_t ps, int m,
              const char *name) {
  if (!X) return fail(MW_EINVAL, "%s is NULL", name);
  if (ld < cols) return fail(MW_EINVAL, "%s: ld %lld < cols %lld", name, (long long)ld, (long long)cols);
  if (m > 1 && ps < rows * ld)
    return fail(MW_EINVAL, "%s: plane stride %lld < rows*ld %lld", name, (long long)ps,
                (long long)(rows * ld));
  return MW_OK;
}

}  // namespace
}  // namespace mw

using namespace mw;

namespace mw {
namespace {

// One CTA waits on a barrier that nothing completes: the bounded wait of the
// pipeline kernels runs out after limit_ns, raises MW_ETIMEOUT and returns.
__global__ void selftest_wait_kernel(uint64_t limit_ns, unsigned int *status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_for(&bar, 0, status, (volatile int *)&abort_flag, limit_ns);
  __syncthreads();
}

}  // namespace
}  // namespace mw

extern "C" {

const char *mw_last_error(void) { return g_msg.c_str(); }

int mw_selftest_timeout(unsigned int limit_us, mw_stream_t stream) {
  if (limit_us < 1 || limit_us > 10000000u) return fail(MW_EINVAL, "limit must be 1 us .. 10 s");
  selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((uint64_t)limit_us * 1000ull,
                                                           status_ptr());
  return cuda_fail(cudaGetLastError(), "self-test launch");
}

const char *mw_version(void) {
  return "mw 0.3 (sm_103a, tcgen05 bf16 slices and residues, fp64 pieces)";
}

int mw_crt_moduli(int *moduli, int n) {
  const int total = crt_table_size();
  if (moduli)
    for (int i = 0; i < n && i < total; ++i) moduli[i] = crt_modulus(i);
  return total;
}

int mw_set_phase_events(void *const *events, int n) {
  if (!events || n <= 0) {
    g_phase_on = false;
    return MW_OK;
  }
  if (n < 4) return fail(MW_EINVAL, "need 4 events");
  for (int i = 0; i < 4; ++i) g_phase[i] = static_cast<cudaEvent_t>(events[i]);
  g_phase_on = true;
  return MW_OK;
}

int mw_get_status(int *bits, int clear) {
  if (!bits) return fail(MW_EINVAL, "bits is NULL");
  unsigned int *p = status_ptr();
  if (!p) return fail(MW_ECUDA, "no status word on this device");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "mw_get_status sync");
  unsigned int v = 0;
  if ((e = cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "mw_get_status read");
  if (clear && (e = cudaMemset(p, 0, sizeof v)) != cudaSuccess)
    return cuda_fail(e, "mw_get_status clear");
  *bits = (int)v;
  return MW_OK;
}

int mw_plan_gemm(int m, int mode, int64_t M, int64_t N, int64_t K, int range_A, int range_B,
                 mw_plan *plan) {
  if (!plan) return fail(MW_EINVAL, "plan is NULL");
  if (!valid_m(m)) return fail(MW_EINVAL, "m = %d, must be 2, 4, 8 or 16", m);
  if (M <= 0 || N <= 0 || K <= 0) return fail(MW_EINVAL, "dimensions must be positive");
  if (range_A < 0 || range_B < 0) return fail(MW_EINVAL, "ranges must be >= 0");
  const int want_w = plan->w;
  // Error budget 2K 2^(-52m) per unit of sum |a||b|, a quarter each to the
  // truncation of A, of B, the dropped pairs and the final rounding:
  //   truncation of A: m 2^(rA + 3 - w S_A) <= K 2^(-52m-1)
  //   dropped pairs:   S_min 2^(rA + rB + 4 - w D) (1 + 2^(1-w)) <= K 2^(-52m-1)
  const double lgK = std::log2((double)K), lgm = std::log2((double)m);
  const double bitsA = 52.0 * m + range_A + lgm + 5.0 - lgK;
  const double bitsB = 52.0 * m + range_B + lgm + 5.0 - lgK;
  mw_plan p{};
  p.m = m;
  p.mode = mode;
  p.range_A = range_A;
  p.range_B = range_B;
  auto finish = [&](int w) {
    p.w = w;
    p.S_A = ceil_div_bits(bitsA, w);
    p.S_B = ceil_div_bits(bitsB, w);
    const int S_min = p.S_A < p.S_B ? p.S_A : p.S_B;
    const double bitsD = 52.0 * m + range_A + range_B + std::log2((double)S_min) + 6.0 - lgK;
    p.D = ceil_div_bits(bitsD, w);
    if (p.D > p.S_A + p.S_B - 1) p.D = p.S_A + p.S_B - 1;
  };
  if (mode == MW_OZAKI) {
    if (want_w != 0 && (want_w < 2 || want_w > 8)) return fail(MW_EINVAL, "Ozaki w must be 2..8");
    finish(want_w ? want_w : 8);
    p.chunk = 1 << (26 - 2 * p.w);  // chunk 2^(2w-2) <= 2^24
    const int S_min = p.S_A < p.S_B ? p.S_A : p.S_B;
    p.group = group_size(S_min, K, p.w);
    if (p.group < 1) return fail(MW_EUNSUPPORTED, "K = %lld too long for 64-bit partial sums", (long long)K);
  } else if (mode == MW_PLAIN) {
    if (m == 16) return fail(MW_EUNSUPPORTED, "m = 16 has no MW_PLAIN form (MW_OZAKI and MW_DOT take it)");
    if (want_w != 0 && (want_w < 4 || want_w > 26)) return fail(MW_EINVAL, "plain w must be 4..26");
    int w = want_w ? want_w : 26;
    for (; w >= 4; --w) {
      finish(w);
      const int S_min = p.S_A < p.S_B ? p.S_A : p.S_B;
      if (std::log2((double)S_min * (double)K) + 2.0 * w - 2.0 <= 53.0) break;
    }
    if (w < 4) return fail(MW_EUNSUPPORTED, "K = %lld too long for exact FP64 sums", (long long)K);
    p.group = 1;
    p.chunk = 0;
  } else if (mode == MW_TEXTBOOK) {
    if (m != 2 && m != 4 && m != 8)
      return fail(MW_EUNSUPPORTED, "the textbook form (MW_TEXTBOOK) takes m = 2, 4 and 8");
    p.w = p.S_A = p.S_B = p.D = p.group = p.chunk = 0;
  } else if (mode == MW_CRT) {
    // fixed-point bits as for the slice form's digits (w = 1: no rounding up to
    // whole digits); no products are dropped, so the moduli only have to hold
    // |X| <= K 2^(L_A + L_B - 2) below P/8
    if (want_w != 0 && want_w != 1) return fail(MW_EINVAL, "MW_CRT plans have w = 1");
    if (m != 2 && m != 4) return fail(MW_EUNSUPPORTED, "the residue form (MW_CRT) takes m = 2 and 4");
    p.w = 1;
    p.S_A = std::max(2, ceil_div_bits(bitsA, 1));
    p.S_B = std::max(2, ceil_div_bits(bitsB, 1));
    if (p.S_A > 381 || p.S_B > 381)
      return fail(MW_EUNSUPPORTED, "MW_CRT: %d / %d fixed-point bits (at most 381)", p.S_A, p.S_B);
    const double need = p.S_A + p.S_B + 1 + lgK;
    int n = 1;
    while (n <= crt_table_size() && crt_bits(n) <= need) ++n;
    if (n > crt_table_size())
      return fail(MW_EUNSUPPORTED, "MW_CRT: the products need %.1f bits, the moduli hold %.1f",
                  need, crt_bits(crt_table_size()));
    p.D = n;
    p.group = 1;
    p.chunk = 0;
  } else if (mode == MW_DOT) {
    if (want_w != 0 && want_w != 24) return fail(MW_EINVAL, "MW_DOT pieces are 24 bits");
    if (M != 1 || N != 1) return fail(MW_EINVAL, "MW_DOT plans one inner product: M = N = 1");
    finish(24);
    int lo = 0, hi = 0;
    dot_pieces_range(m, &lo, &hi);
    const int S = std::max(std::max(p.S_A, p.S_B), lo);
    if (S > hi) return fail(MW_EUNSUPPORTED, "inner products need %d pieces, at most %d", S, hi);
    p.S_A = p.S_B = S;
    const double bitsD = 52.0 * m + range_A + range_B + std::log2((double)S) + 6.0 - lgK;
    p.D = std::min(ceil_div_bits(bitsD, 24), 2 * S - 1);
    if (p.D > S + 4) return fail(MW_EUNSUPPORTED, "inner products keep at most S + 4 diagonals");
    // a thread's int64 diagonal sums take ceil(K / 256) products below 2^46 each
    if ((double)S * std::ceil((double)K / 256.0) > std::ldexp(1.0, 16))
      return fail(MW_EUNSUPPORTED, "K = %lld too long for the inner-product kernel", (long long)K);
    p.group = 1;
    p.chunk = 0;
  } else {
    return fail(MW_EINVAL, "mode must be MW_PLAIN, MW_OZAKI, MW_CRT, MW_TEXTBOOK or MW_DOT");
  }
  *plan = p;
  return MW_OK;
}

int mw_split(int m, int trans, int64_t R, int64_t K, const double *X, int64_t ld,
             int64_t plane_stride, int w, int S, int format, void *digits, int64_t digit_ld,
             int32_t *exps, int32_t *spread, int32_t *max_spread, int range, mw_stream_t stream) {
  if (!valid_m(m)) return fail(MW_EINVAL, "m = %d, must be 2, 4, 8 or 16", m);
  if (R <= 0 || K <= 0) return fail(MW_EINVAL, "dimensions must be positive");
  int rc = trans ? check_mat(X, K, R, ld, plane_stride, m, "X") : check_mat(X, R, K, ld, plane_stride, m, "X");
  if (rc) return rc;
  if (!digits || !exps) return fail(MW_EINVAL, "digits/exps is NULL");
  if (digit_ld < K || digit_ld % 64) return fail(MW_EINVAL, "digit_ld must be >= K and a multiple of 64");
  if (w < 2 || w > 26 || S < 1) return fail(MW_EINVAL, "bad w or S");
  if (format == MW_DIGITS_BF16 && w > 9) return fail(MW_EINVAL, "bfloat16 pieces need w <= 9");
  if (format != MW_DIGITS_BF16 && format != MW_DIGITS_F64) return fail(MW_EINVAL, "bad format");
  if (!spread) return fail(MW_EINVAL, "spread is NULL");
  SplitArgs a{};
  a.m = m; a.trans = trans; a.w = w; a.S = S; a.format = format; a.range = range;
  a.R = R; a.K = K; a.ld = ld; a.plane_stride = plane_stride; a.digit_ld = digit_ld;
  a.X = X; a.digits = digits; a.exps = exps; a.spread = spread; a.max_spread = max_spread;
  rc = launch_split(a, false, (cudaStream_t)stream);
  return rc;
}

int mw_gemm_workspace_size(const mw_plan *plan, int64_t M, int64_t N, int64_t K, size_t *bytes) {
  if (!bytes) return fail(MW_EINVAL, "bytes is NULL");
  int rc = check_plan(plan, M, N, K);
  if (rc) return rc;
  *bytes = layout(*plan, M, N, K).total;
  return MW_OK;
}

int mw_gemm_workspace_layout(const mw_plan *plan, int64_t M, int64_t N, int64_t K,
                             size_t offsets[4], size_t *bytes) {
  if (!offsets || !bytes) return fail(MW_EINVAL, "offsets/bytes is NULL");
  int rc = check_plan(plan, M, N, K);
  if (rc) return rc;
  const Layout L = layout(*plan, M, N, K);
  offsets[0] = L.exps;
  offsets[1] = L.digA;
  offsets[2] = L.digB;
  offsets[3] = L.partials;
  *bytes = L.total;
  return MW_OK;
}

namespace {

struct Operands {
  int32_t *eA, *spA, *eB, *spB, *maxsp, *redo;
};

Operands ops_in(void *ws, int64_t M, int64_t N) {
  int32_t *base = static_cast<int32_t *>(ws);
  Operands o;
  o.eA = base;
  o.spA = base + M;
  o.eB = base + 2 * M;
  o.spB = base + 2 * M + N;
  o.maxsp = base + 2 * M + 2 * N;
  o.redo = base + 2 * M + 2 * N + 2;
  return o;
}

// A second stream per device: op(B) is cut there while op(A) is cut on the
// caller's stream (the two splits share nothing); events fork and join the two,
// which also holds inside a stream capture.
cudaStream_t side_stream() {
  static cudaStream_t st[kMaxDevices] = {nullptr};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_status_mu);
  if (!st[dev] && cudaStreamCreateWithFlags(&st[dev], cudaStreamNonBlocking) != cudaSuccess)
    st[dev] = nullptr;
  return st[dev];
}

int split_both(const mw_plan &p, int transA, int transB, int64_t M, int64_t N, int64_t K,
               const double *A, int64_t lda, int64_t psa, const double *B, int64_t ldb,
               int64_t psb, void *ws, const Layout &L, bool exps_only, cudaStream_t s) {
  // residue splits hold tensor memory on every SM they run on: with more than
  // 64 moduli two of them would not fit side by side, so they run one after the
  // other on the caller's stream
  cudaStream_t s2 = (p.mode == MW_CRT && !exps_only && p.D > 64) ? nullptr : side_stream();
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool fork = s2 != nullptr &&
              cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) == cudaSuccess;
  if (fork) fork = cudaEventRecord(ev[0], s) == cudaSuccess &&
                   cudaStreamWaitEvent(s2, ev[0], 0) == cudaSuccess;
  if (!fork) s2 = s;
  Operands o = ops_in(ws, M, N);
  uint8_t *w8 = static_cast<uint8_t *>(ws);
  SplitArgs a{};
  a.m = p.m; a.w = p.w; a.format = p.mode == MW_PLAIN ? MW_DIGITS_F64 : MW_DIGITS_BF16;
  a.nmod = p.mode == MW_CRT ? p.D : 0;
  a.K = K; a.digit_ld = L.Kp;
  // op(A): rows M; stored M x K (trans 0) or K x M (trans 1)
  a.trans = transA; a.R = M; a.ld = lda; a.plane_stride = psa; a.X = A; a.S = p.S_A;
  a.digits = w8 + L.digA; a.exps = o.eA; a.spread = o.spA; a.max_spread = o.maxsp;
  a.range = p.range_A;
  a.redo = p.mode == MW_CRT ? o.redo : nullptr;
  int rc = launch_split(a, exps_only, s);
  if (!rc) {
    // op(B) used as its transpose: rows N; B stored K x N (trans 0 -> columns) or N x K
    a.trans = !transB; a.R = N; a.ld = ldb; a.plane_stride = psb; a.X = B; a.S = p.S_B;
    a.digits = w8 + L.digB; a.exps = o.eB; a.spread = o.spB; a.max_spread = o.maxsp + 1;
    a.range = p.range_B;
    a.redo = p.mode == MW_CRT ? o.redo + 1 : nullptr;
    rc = launch_split(a, exps_only, s2);
  }
  // join the side stream whatever happened (inside a capture a fork must be joined)
  if (fork) {
    cudaError_t e = cudaEventRecord(ev[1], s2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[1], 0);
    if (e != cudaSuccess && !rc) rc = cuda_fail(e, "split join");
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);   // released once the recorded work is done
  return rc;
}

int check_gemm_mats(int m, int transA, int transB, int64_t M, int64_t N, int64_t K,
                    const double *A, int64_t lda, int64_t psa, const double *B, int64_t ldb,
                    int64_t psb) {
  int rc = transA ? check_mat(A, K, M, lda, psa, m, "A") : check_mat(A, M, K, lda, psa, m, "A");
  if (rc) return rc;
  return transB ? check_mat(B, N, K, ldb, psb, m, "B") : check_mat(B, K, N, ldb, psb, m, "B");
}

}  // namespace

int mw_gemm(const mw_plan *plan, int transA, int transB, int64_t M, int64_t N, int64_t K,
            const double *A, int64_t lda, int64_t psa, const double *B, int64_t ldb, int64_t psb,
            double *C, int64_t ldc, int64_t psc, void *ws, size_t ws_bytes, mw_stream_t stream) {
  int rc = check_plan(plan, M, N, K);
  if (rc) return rc;
  const mw_plan &p = *plan;
  if ((rc = check_gemm_mats(p.m, transA, transB, M, N, K, A, lda, psa, B, ldb, psb))) return rc;
  if ((rc = check_mat(C, M, N, ldc, psc, p.m, "C"))) return rc;
  const Layout L = layout(p, M, N, K);
  if (!ws || ws_bytes < L.total)
    return fail(MW_ENOSPC, "workspace %zu bytes, need %zu", ws_bytes, L.total);
  cudaStream_t s = (cudaStream_t)stream;
  if (p.mode == MW_TEXTBOOK) {
    phase(0, s);
    phase(1, s);
    rc = launch_textbook(p.m, transA, transB, M, N, K, A, lda, psa, B, ldb, psb, C, ldc, psc, s);
    phase(2, s);
    phase(3, s);
    return rc;
  }
  phase(0, s);
  cudaError_t e = cudaMemsetAsync(ops_in(ws, M, N).maxsp, 0, 2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "mw_gemm memset");
  if ((rc = split_both(p, transA, transB, M, N, K, A, lda, psa, B, ldb, psb, ws, L, false, s)))
    return rc;
  phase(1, s);
  Operands o = ops_in(ws, M, N);
  uint8_t *w8 = static_cast<uint8_t *>(ws);
  if (p.mode == MW_PLAIN) {
    PlainArgs a{};
    a.m = p.m; a.w = p.w; a.S_A = p.S_A; a.S_B = p.S_B; a.D = p.D;
    a.M = M; a.N = N; a.Kp = L.Kp;
    a.dA = reinterpret_cast<const double *>(w8 + L.digA);
    a.dB = reinterpret_cast<const double *>(w8 + L.digB);
    a.eA = o.eA; a.eB = o.eB; a.C = C; a.ldc = ldc; a.psc = psc;
    rc = launch_plain(a, s);
    phase(2, s);
    phase(3, s);
    return rc;
  }
  OzakiArgs a{};
  a.m = p.m; a.w = p.w; a.S_A = p.S_A; a.S_B = p.S_B; a.D = p.D; a.group = p.group;
  a.chunk = p.chunk; a.M = M; a.N = N; a.Kp = L.Kp;
  a.crt = p.mode == MW_CRT;
  a.dA = w8 + L.digA; a.dB = w8 + L.digB; a.eA = o.eA; a.eB = o.eB;
  a.partials = w8 + L.partials;
  a.C = C; a.ldc = ldc; a.psc = psc;
  rc = launch_ozaki(a, s, [&] { phase(2, s); });
  phase(3, s);
  return rc;
}

int mw_elementwise(int op, int m, int64_t n, const double *A, int64_t plane_stride_a,
                   const double *B, int64_t plane_stride_b, double *C, int64_t plane_stride_c,
                   mw_stream_t stream) {
  if (op != MW_OP_ADD && op != MW_OP_MUL && op != MW_OP_DIV)
    return fail(MW_EINVAL, "mw_elementwise: op %d (add 0, mul 1, div 2)", op);
  if (m != 2 && m != 4 && m != 8) return fail(MW_EINVAL, "mw_elementwise: m = %d (2, 4 or 8)", m);
  if (n < 0) return fail(MW_EINVAL, "mw_elementwise: n = %lld", (long long)n);
  if (n == 0) return MW_OK;
  if (!A || !B || !C) return fail(MW_EINVAL, "mw_elementwise: NULL operand");
  if (plane_stride_a < n || plane_stride_b < n || plane_stride_c < n)
    return fail(MW_EINVAL, "mw_elementwise: plane strides must be at least n");
  return launch_elementwise(op, m, n, A, plane_stride_a, B, plane_stride_b, C, plane_stride_c,
                            (cudaStream_t)stream);
}

int mw_measure_spread(int m, int transA, int transB, int64_t M, int64_t N, int64_t K,
                      const double *A, int64_t lda, int64_t psa, const double *B, int64_t ldb,
                      int64_t psb, void *ws, size_t ws_bytes, int *range_A, int *range_B,
                      mw_stream_t stream) {
  if (!valid_m(m)) return fail(MW_EINVAL, "m = %d, must be 2, 4, 8 or 16", m);
  if (M <= 0 || N <= 0 || K <= 0) return fail(MW_EINVAL, "dimensions must be positive");
  if (!range_A || !range_B) return fail(MW_EINVAL, "range outputs are NULL");
  int rc = check_gemm_mats(m, transA, transB, M, N, K, A, lda, psa, B, ldb, psb);
  if (rc) return rc;
  const size_t need = sizeof(int32_t) * (2 * (size_t)M + 2 * (size_t)N + 2);
  if (!ws || ws_bytes < need) return fail(MW_ENOSPC, "workspace %zu bytes, need %zu", ws_bytes, need);
  mw_plan p{};
  p.m = m; p.mode = MW_PLAIN; p.w = 20; p.S_A = p.S_B = 1; p.D = 1;
  p.range_A = p.range_B = -1;
  Layout L{};
  L.Kp = round_up(K, 64);
  cudaStream_t s = (cudaStream_t)stream;
  Operands o = ops_in(ws, M, N);
  cudaError_t e = cudaMemsetAsync(o.maxsp, 0, 2 * sizeof(int32_t), s);
  if (e != cudaSuccess) return cuda_fail(e, "measure memset");
  if ((rc = split_both(p, transA, transB, M, N, K, A, lda, psa, B, ldb, psb, ws, L, true, s)))
    return rc;
  int32_t host[2];
  if ((e = cudaMemcpyAsync(host, o.maxsp, sizeof host, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "measure read");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "measure sync");
  *range_A = host[0];
  *range_B = host[1];
  return MW_OK;
}

int mw_gemm_backward(const mw_plan *plan_dA, const mw_plan *plan_dB, int64_t M, int64_t N,
                     int64_t K, const double *A, int64_t lda, int64_t psa, const double *B,
                     int64_t ldb, int64_t psb, const double *G, int64_t ldg, int64_t psg,
                     double *dA, int64_t ldda, int64_t psda, double *dB, int64_t lddb,
                     int64_t psdb, void *ws, size_t ws_bytes, mw_stream_t stream) {
  int rc;
  if (dA) {
    // dA (M x K) = G (M x N) B^T, B stored K x N: reduction over N
    if ((rc = mw_gemm(plan_dA, 0, 1, M, K, N, G, ldg, psg, B, ldb, psb, dA, ldda, psda, ws,
                      ws_bytes, stream)))
      return rc;
  }
  if (dB) {
    // dB (K x N) = A^T (K x M) G (M x N), A stored M x K: reduction over M
    if ((rc = mw_gemm(plan_dB, 1, 0, K, N, M, A, lda, psa, G, ldg, psg, dB, lddb, psdb, ws,
                      ws_bytes, stream)))
      return rc;
  }
  return MW_OK;
}

}  // extern "C"
