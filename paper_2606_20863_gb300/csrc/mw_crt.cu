// MW_CRT: the residue form of the product (the second Ozaki scheme, which
// Sections 1 and 4 point to as the tensor-core route for the error-free
// summation).
//
// Steps 1-2 stay those of Section 2: one shared exponent per row of op(A) and
// column of op(B), every word truncated on the fixed-point grid of L bits,
//   T = sum_j trunc(x_j 2^(L - 2 - E)),   -2^(L-1) <= T < 2^(L-1).
// Instead of cutting T into w-bit digits and multiplying every pair of digit
// matrices, T is reduced modulo n small pairwise coprime moduli p_i (balanced
// residues, at most floor(p_i / 2) <= 256 in magnitude, so exact in bfloat16),
// and one tensor-core product per modulus gives the exact integer sums
//   Y_i = sum_k r^A_i,k r^B_i,k            (mw_ozaki.cu, its CRT instance).
// The exact product X = sum_k T^A_k T^B_k is the unique integer in (-P/2, P/2]
// with X = Y_i mod p_i, P = p_1 ... p_n > 8 max|X| (Chinese remainder theorem):
//   y_i = Y_i (P/p_i)^(-1) mod p_i,   X = sum_i y_i (P/p_i) - k P,
// k = round(sum_i y_i / p_i), exact because |X| < P/8 leaves the fractional part
// of sum_i y_i / p_i within 1/8 of an integer and the float sum errs by far
// less.  X 2^(E_A + E_B + 4 - L_A - L_B) is rounded into m words greedily
// (round_column), as in the slice form.
//
// This file holds the table of moduli, the residue split and the
// reconstruction; the product kernel is the slice form's, one pair per modulus.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "mw_column.cuh"
#include "mw_device.cuh"
#include "mw_internal.h"
#include "mw_pieces.cuh"

namespace mw {
namespace {

// Pairwise coprime moduli, at most 513 (balanced residues within bfloat16's
// exact integers).  The set: greedy from 363 downwards (keep a number when it
// is coprime to every number kept), then every prime in 364..513.  The order:
// by bits per tensor-core product, log2(p), divided by 1.15 for the moduli
// above 363, whose products need a drain every 64 products (a drain is due
// before chunk * floor(p/2)^2 passes 2^22: 256 products for p <= 257, 128 for
// p <= 363, 64 for p <= 513).  A product uses the first n moduli.
constexpr uint16_t kModuli[] = {
    363, 362, 361, 359, 355, 353, 349, 347, 343, 337, 331, 317, 313, 311, 307, 299,
    293, 289, 283, 281, 277, 271, 269, 263, 257, 251, 241, 239, 233, 229, 227, 509,
    503, 223, 499, 491, 487, 479, 211, 467, 463, 461, 457, 449, 443, 199, 439, 197,
    433, 431, 193, 421, 191, 419, 409, 401, 397, 179, 389, 383, 379, 173, 373, 367,
    167, 163, 157, 151, 149, 139, 137, 131, 127, 113, 109, 107, 103, 101, 97,  89,
    83,  79,  73,  67,  61,  59,  53,  47,  43,  41,  37,  31,  29};
constexpr int kNumModuli = sizeof(kModuli) / sizeof(kModuli[0]);
static_assert(kNumModuli <= kCrtMaxModuli, "moduli table too long");
constexpr int kPow16 = 65;   // 2^(16 j) mod p for j = 0..64 (T of up to 16 64-bit limbs)

// Per modulus: p, floor(2^32 / p) for reducing 32-bit values, 2^(16 j) mod p.
struct CrtTab {
  uint32_t p[kCrtMaxModuli];
  uint32_t m32[kCrtMaxModuli];
  uint32_t pow16[kCrtMaxModuli][kPow16];
};
constexpr CrtTab make_crt_tab() {
  CrtTab t{};
  for (int i = 0; i < kNumModuli; ++i) {
    const uint32_t p = kModuli[i];
    t.p[i] = p;
    t.m32[i] = (uint32_t)((1ull << 32) / p);
    uint32_t x = 1u % p;
    for (int j = 0; j < kPow16; ++j) {
      t.pow16[i][j] = x;
      x = (uint32_t)((uint64_t)x * 65536u % p);
    }
  }
  return t;
}
__constant__ CrtTab kCrt = make_crt_tab();

// x mod p for any 32-bit x: q = floor(x m32 / 2^32) is floor(x/p) or one less.
__device__ __forceinline__ uint32_t mod_u32(uint32_t x, uint32_t p, uint32_t m32) {
  uint32_t r = x - __umulhi(x, m32) * p;
  return r >= p ? r - p : r;
}

// The residue of T in [-floor(p/2), ceil(p/2) - 1]: r >= p - floor(p/2) maps to r - p.
__device__ __forceinline__ int balanced(uint32_t r, uint32_t p) {
  return r >= p - (p >> 1) ? (int)r - (int)p : (int)r;
}

// T in [-2^(L-1), 2^(L-1)): every bit from L-1 up equals the sign.
template <int NL>
__device__ __forceinline__ bool in_range_bits(const uint64_t (&T)[NL], int L) {
  const int b = L - 1, lb = b >> 6, ob = b & 63;
  int64_t v = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i)
    if (i == lb) v = (int64_t)T[i] >> ob;
  bool ok = (v == 0 || v == -1) && lb < NL;
#pragma unroll
  for (int i = 0; i < NL; ++i)
    if (i > lb) ok &= T[i] == (uint64_t)v;
  return ok;
}

// Balanced residues of two fixed-point values (entries k, k+1 of one row)
// modulo the first nmod moduli, stored as bfloat16 pairs in planes 0..nmod-1.
// T = sum_j v_j 2^(16 j) - s 2^(64 NL) with 16-bit pieces v_j and the sign s,
// so T mod p = sum_j v_j (2^(16j) mod p) + s (p - 2^(64 NL) mod p), a sum below
// 64 NL 2^25 + 2^9 <= 2^32 for NL <= 16.
template <int MW, int NL>
__device__ __forceinline__ void residue_pair(const double (&w0)[MW], const double (&w1)[MW], int F,
                                             int L, int nmod, __nv_bfloat16 *dst, int64_t plane,
                                             unsigned int *status) {
  uint64_t T0[NL], T1[NL];
  fixed_point<MW, NL>(w0, F, T0);
  fixed_point<MW, NL>(w1, F, T1);
  if (!(in_range_bits<NL>(T0, L) && in_range_bits<NL>(T1, L))) raise_status(status, MW_ERANGE);
  const bool n0 = (int64_t)T0[NL - 1] < 0, n1 = (int64_t)T1[NL - 1] < 0;
  uint32_t v0[4 * NL], v1[4 * NL];
#pragma unroll
  for (int l = 0; l < NL; ++l)
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      v0[4 * l + h] = (uint32_t)(T0[l] >> (16 * h)) & 0xFFFFu;
      v1[4 * l + h] = (uint32_t)(T1[l] >> (16 * h)) & 0xFFFFu;
    }
  for (int i = 0; i < nmod; ++i) {
    const uint32_t p = kCrt.p[i], m32 = kCrt.m32[i];
    const uint32_t top = p - kCrt.pow16[i][4 * NL];
    uint32_t s0 = n0 ? top : 0u, s1 = n1 ? top : 0u;
#pragma unroll
    for (int j = 0; j < 4 * NL; ++j) {
      const uint32_t c = kCrt.pow16[i][j];
      s0 += v0[j] * c;
      s1 += v1[j] * c;
    }
    const int r0 = balanced(mod_u32(s0, p, m32), p), r1 = balanced(mod_u32(s1, p, m32), p);
    *reinterpret_cast<uint32_t *>(dst + (int64_t)i * plane) =
        (uint32_t)small_int_bf16(r0) | ((uint32_t)small_int_bf16(r1) << 16);
  }
}

// trans = 0: one thread per (row, pair of columns), pairs over the padded width.
template <int MW, int NL>
__global__ void residues_rows_kernel(const double *__restrict__ X, int64_t R, int64_t K, int64_t ld,
                                     int64_t ps, int L, int nmod, __nv_bfloat16 *res,
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
  residue_pair<MW, NL>(a, b, L - 2 - E[r], L, nmod, res + r * dld + k, R * dld, status);
}

// trans = 1: 32 x 32 tiles (32 rows r, 32 columns k of the logical operand)
// staged through shared memory, then reduced like trans = 0.
template <int MW, int NL>
__global__ void residues_cols_kernel(const double *__restrict__ X, int64_t R, int64_t K, int64_t ld,
                                     int64_t ps, int L, int nmod, __nv_bfloat16 *res,
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
    residue_pair<MW, NL>(a, b, L - 2 - E[r], L, nmod, res + r * dld + k, R * dld, status);
  }
}

template <int MW, int NL>
int launch_residues_t(const SplitArgs &a, cudaStream_t s) {
  auto *res = static_cast<__nv_bfloat16 *>(a.digits);
  if (!a.trans) {
    const int64_t n = a.R * (a.digit_ld / 2);
    const int threads = 256;
    residues_rows_kernel<MW, NL><<<(unsigned)((n + threads - 1) / threads), threads, 0, s>>>(
        a.X, a.R, a.K, a.ld, a.plane_stride, a.S, a.nmod, res, a.digit_ld, a.exps, status_ptr());
  } else {
    dim3 grid((unsigned)((a.R + 31) / 32), (unsigned)((a.digit_ld + 31) / 32));
    const size_t sm = (size_t)MW * 32 * 33 * sizeof(double);
    static bool attr_set = false;  // once per instantiation
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(residues_cols_kernel<MW, NL>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return cuda_fail(e, "residue split smem attribute");
      attr_set = true;
    }
    residues_cols_kernel<MW, NL><<<grid, dim3(32, 8), sm, s>>>(
        a.X, a.R, a.K, a.ld, a.plane_stride, a.S, a.nmod, res, a.digit_ld, a.exps, status_ptr());
  }
  return cuda_fail(cudaGetLastError(), "residue split launch");
}

template <int MW>
int launch_residues_nl(const SplitArgs &a, cudaStream_t s) {
  const int bits = a.S + 3;    // |T| < m 2^(L-2) < 2^(L+1), one sign bit
  if (bits <= 128) return launch_residues_t<MW, 2>(a, s);
  if (bits <= 256) return launch_residues_t<MW, 4>(a, s);
  if (bits <= 384) return launch_residues_t<MW, 6>(a, s);
  return fail(MW_EUNSUPPORTED, "residue form: %d fixed-point bits (at most 381)", a.S);
}

// ---- reconstruction -----------------------------------------------------------
// Constants of the first D moduli, computed on the host for every launch and
// passed by value (kernel parameters, so that a captured launch keeps them).
struct CrtFuse {
  int D, pad;
  uint32_t p[kCrtMaxModuli], m32[kCrtMaxModuli], inv[kCrtMaxModuli], c31[kCrtMaxModuli];
  float rcp[kCrtMaxModuli];
  uint32_t Q[kCrtMaxModuli][kCrtMaxLimbs];   // P / p_i, 32-bit limbs
  uint32_t P[kCrtMaxLimbs];
};

// One thread per output (i along the column-major planes): Y_t -> y_t ->
// X = sum_t y_t Q_t - k P in NL32 32-bit limbs (two's complement, mod 2^(32 NL32),
// enough for |X| < P/8), then the greedy words of X 2^(E_i + E_j + ex0).
template <int MW, int NL32>
__global__ void __launch_bounds__(128) crt_combine_kernel(
    const int32_t *__restrict__ partials, const int32_t *eA, const int32_t *eB, int64_t M,
    int64_t N, int ex0, double *C, int64_t ldc, int64_t psc, const __grid_constant__ CrtFuse F) {
  __shared__ uint32_t limbs[NL32][128];
  const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x, j = blockIdx.y;
  if (i >= M || j >= N) return;
  uint64_t acc[NL32];
#pragma unroll
  for (int l = 0; l < NL32; ++l) acc[l] = 0;
  float kf = 0.f;
  const int32_t *y_in = partials + j * M + i;
  const int64_t plane = M * N;
  int32_t nxt = y_in[0];
  for (int t = 0; t < F.D; ++t) {
    const int32_t v = nxt;
    if (t + 1 < F.D) nxt = y_in[(t + 1) * plane];
    const uint32_t p = F.p[t], m32 = F.m32[t];
    // v mod p from v + 2^31 >= 0, then y = v (P/p)^(-1) mod p
    int r = (int)mod_u32((uint32_t)v ^ 0x80000000u, p, m32) - (int)F.c31[t];
    if (r < 0) r += (int)p;
    const uint32_t y = mod_u32((uint32_t)r * F.inv[t], p, m32);
    kf = fmaf((float)y, F.rcp[t], kf);
#pragma unroll
    for (int l = 0; l < NL32; ++l) acc[l] += (uint64_t)y * F.Q[t][l];
  }
  const uint32_t k = (uint32_t)rintf(kf);
  uint32_t U[NL32];
  uint64_t carry = 0, mc = 0;
  uint32_t br = 0;
#pragma unroll
  for (int l = 0; l < NL32; ++l) {
    const uint64_t s = acc[l] + carry;
    carry = s >> 32;
    const uint64_t kp = (uint64_t)k * F.P[l] + mc;
    mc = kp >> 32;
    const uint64_t d = (uint64_t)(uint32_t)s - (uint32_t)kp - br;
    U[l] = (uint32_t)d;
    br = (uint32_t)(d >> 63);
  }
  double *c = C + i * ldc + j;
  round_column<MW, NL32>(U, &limbs[0][threadIdx.x], 128, eA[i] + eB[j] + ex0,
                         [&](int w, double x) { c[w * psc] = x; });
}

// ---- host arithmetic on the constants ------------------------------------------
using Big = std::vector<uint32_t>;   // little-endian 32-bit limbs

void big_mul_small(Big &x, uint32_t a) {
  uint64_t c = 0;
  for (uint32_t &v : x) {
    const uint64_t s = (uint64_t)v * a + c;
    v = (uint32_t)s;
    c = s >> 32;
  }
  if (c) x.push_back((uint32_t)c);
}
uint32_t big_div_small(const Big &x, uint32_t a, Big *q) {   // returns x mod a
  uint64_t r = 0;
  if (q) q->assign(x.size(), 0);
  for (size_t i = x.size(); i-- > 0;) {
    const uint64_t cur = (r << 32) | x[i];
    if (q) (*q)[i] = (uint32_t)(cur / a);
    r = cur % a;
  }
  return (uint32_t)r;
}
uint32_t inverse_mod(uint32_t a, uint32_t p) {   // a^(-1) mod p, gcd(a, p) = 1
  int64_t t = 0, nt = 1, r = p, nr = a % p;
  while (nr) {
    const int64_t q = r / nr;
    int64_t tmp = t - q * nt; t = nt; nt = tmp;
    tmp = r - q * nr; r = nr; nr = tmp;
  }
  return (uint32_t)(t < 0 ? t + p : t);
}

template <int MW, int NL32>
int launch_crt_combine_t(const OzakiArgs &a, const CrtFuse &F, cudaStream_t s) {
  dim3 grid((unsigned)((a.M + 127) / 128), (unsigned)a.N);
  crt_combine_kernel<MW, NL32><<<grid, 128, 0, s>>>(
      static_cast<const int32_t *>(a.partials), a.eA, a.eB, a.M, a.N, 4 - a.S_A - a.S_B, a.C,
      a.ldc, a.psc, F);
  return cuda_fail(cudaGetLastError(), "residue reconstruction launch");
}

template <int MW>
int launch_crt_combine_m(const OzakiArgs &a, const CrtFuse &F, int bitsP, cudaStream_t s) {
  const int need = bitsP + 1;   // |X| < P/8 < 2^bitsP, and a sign bit
  if (need <= 256) return launch_crt_combine_t<MW, 8>(a, F, s);
  if (need <= 384) return launch_crt_combine_t<MW, 12>(a, F, s);
  if (need <= 512) return launch_crt_combine_t<MW, 16>(a, F, s);
  if (need <= 640) return launch_crt_combine_t<MW, 20>(a, F, s);
  if (need <= 768) return launch_crt_combine_t<MW, 24>(a, F, s);
  return fail(MW_EUNSUPPORTED, "residue form: modulus product of %d bits", bitsP);
}

}  // namespace

int crt_table_size() { return kNumModuli; }
int crt_modulus(int i) { return (i >= 0 && i < kNumModuli) ? kModuli[i] : 0; }
int crt_chunk(int i) {
  const int h = crt_modulus(i) / 2;
  return h * h <= (1 << 14) ? 256 : h * h <= (1 << 15) ? 128 : 64;
}
double crt_bits(int n) {
  double b = 0;
  for (int i = 0; i < n && i < kNumModuli; ++i) b += std::log2((double)kModuli[i]);
  return b;
}

int launch_residues(const SplitArgs &a, cudaStream_t s) {
  if (a.nmod < 1 || a.nmod > kNumModuli)
    return fail(MW_EINVAL, "residue form: %d moduli (1..%d)", a.nmod, kNumModuli);
  switch (a.m) {
    case 2: return launch_residues_nl<2>(a, s);
    case 4: return launch_residues_nl<4>(a, s);
  }
  return fail(MW_EUNSUPPORTED, "residue form: m = %d (2 or 4)", a.m);
}

int launch_crt_combine(const OzakiArgs &a, cudaStream_t s) {
  const int D = a.D;
  if (D < 1 || D > kNumModuli) return fail(MW_EINVAL, "residue form: %d moduli", D);
  CrtFuse F{};
  F.D = D;
  Big P{1};
  for (int t = 0; t < D; ++t) big_mul_small(P, kModuli[t]);
  if ((int)P.size() > kCrtMaxLimbs) return fail(MW_EUNSUPPORTED, "modulus product too long");
  for (int t = 0; t < D; ++t) {
    const uint32_t p = kModuli[t];
    Big Q;
    big_div_small(P, p, &Q);
    const uint32_t qm = big_div_small(Q, p, nullptr);
    F.p[t] = p;
    F.m32[t] = (uint32_t)((1ull << 32) / p);
    F.inv[t] = inverse_mod(qm, p);
    F.c31[t] = (uint32_t)((1ull << 31) % p);
    F.rcp[t] = 1.0f / (float)p;
    for (int l = 0; l < kCrtMaxLimbs; ++l) F.Q[t][l] = l < (int)Q.size() ? Q[l] : 0u;
  }
  for (int l = 0; l < kCrtMaxLimbs; ++l) F.P[l] = l < (int)P.size() ? P[l] : 0u;
  const int bitsP = (int)std::ceil(crt_bits(D));
  switch (a.m) {
    case 2: return launch_crt_combine_m<2>(a, F, bitsP, s);
    case 4: return launch_crt_combine_m<4>(a, F, bitsP, s);
  }
  return fail(MW_EUNSUPPORTED, "residue form: m = %d (2 or 4)", a.m);
}

}  // namespace mw
