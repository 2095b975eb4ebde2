/* mw.h -- C interface of the GB300 m-double matrix product library (libmw.so).
 *
 * An m-double is an unevaluated sum of m nonoverlapping doubles (Section 1 of
 * J. Verschelde, "Multiword Arithmetic and Parallel Computing"); m is 2
 * (double double), 4 (quad double), 8 (octo double) or 16 (hexa double,
 * Table 2's 16d precision; MW_OZAKI single products and mw_dot_batched only,
 * not MW_PLAIN nor batches).  A matrix of
 * m-doubles is stored as m planes of doubles ("structure of arrays", the
 * register-friendly layout the abstract argues for): entry (r, c) of word
 * plane j is at  base[j * plane_stride + r * ld + c]  (row major, ld >= cols,
 * plane_stride >= rows * ld, planes must not overlap).
 *
 * The library computes C = op(A) op(B) with the paper's error-free
 * summation (Section 2, Figure 1; matrix form in Section 4):
 *   1. every row of op(A) and every column of op(B) gets one shared exponent E;
 *   2. every entry is cut, on a fixed-point grid below 2^E, into S pieces of w
 *      bits whose high bits are zero (balanced digits, |d| <= 2^(w-1));
 *   3. the products of pieces are summed exactly, grouped by diagonal
 *      t = p + q, s_t = sum_{p+q=t} sum_k dA_{p,ik} dB_{q,kj}  (the paper's s_i);
 *   4. the diagonal sums are fused into m nonoverlapping doubles.
 * Two forms compute step 3:
 *   MW_PLAIN  pieces are doubles (w about 20), products and sums on the FP64
 *             pipe, exact while the number of terms stays below the threshold
 *             of Section 2; step 4 adds the scaled s_t in m-double arithmetic.
 *   MW_OZAKI  pieces are integers of w = 7 or 8 bits held in bfloat16, every
 *             pair of piece matrices is a tensor-core product (tcgen05,
 *             fp32 accumulation, exact below 2^24 and drained to 64-bit integers
 *             before that), the "stepping stone to the Ozaki scheme" of
 *             Section 1; step 4 is exact integer fusion and rounding to nearest
 *             of each word in turn.
 *   MW_CRT    the residue form (the second Ozaki scheme): the same fixed-point
 *             integers T of step 2, reduced modulo n small pairwise coprime
 *             moduli (balanced residues, exact in bfloat16); one tensor-core
 *             product per modulus gives every sum of products mod p_i, and the
 *             Chinese remainder theorem rebuilds the exact integer products,
 *             which step 4 rounds as in MW_OZAKI.  n grows with the bits of
 *             T_A + T_B, where MW_OZAKI's pair count grows with their square
 *             (m = 2 and 4).
 * and a reference form without error-free summation:
 *   MW_TEXTBOOK the "ordinary" product Table 2 compares against: every term an
 *             m-double multiplication and addition (two_sum, two_prod, m-word
 *             renormalisation) on the FP64 pipe, k in order (m = 2, 4, 8; no
 *             workspace beyond 256 bytes; the plan fixes only m and the form).
 * Inner products (mw_dot_batched, the workload of Table 2) use a fourth form:
 *   MW_DOT    pieces are 24-bit integers, products summed in int64 on the
 *             integer units (no operand reuse, so no tensor cores); exact
 *             integer fusion and rounding as for MW_OZAKI.
 *
 * Conventions for every entry point:
 *  - Device pointers unless the name says otherwise; the caller owns all memory.
 *  - Work is ordered on `stream` (a cudaStream_t; NULL = legacy default stream)
 *    and is asynchronous unless the comment says the call synchronizes.
 *  - The return value is MW_OK or an MW_E* code for errors found on the host
 *    (bad arguments, launch failures).  Errors found on the GPU (non-finite or
 *    badly normalised input, a wait that timed out) are OR-ed into a per-device
 *    status word that mw_get_status() reads.
 *  - mw_last_error() gives a message for the last host-side error of the
 *    calling thread.  Nothing throws across this interface.
 */
#ifndef MW_H
#define MW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mw_stream_t; /* same type as cudaStream_t */

/* return codes (host) and status bits (device, see mw_get_status) */
enum {
  MW_OK = 0,
  MW_EINVAL = 1,      /* bad argument: m not in {2,4,8,16} (or 16 where the form takes
                         only {2,4,8}), dims <= 0, ld too small, NULL */
  MW_ERANGE = 2,      /* status bit: fixed-point value outside [-2^(wS-1), 2^(wS-1)) (input not normalised) */
  MW_ENONFINITE = 4,  /* status bit: an input word is inf or nan */
  MW_ECUDA = 8,       /* a CUDA call failed */
  MW_ETIMEOUT = 16,   /* status bit: a bounded wait inside a kernel gave up */
  MW_ENOSPC = 32,     /* workspace smaller than mw_gemm_workspace_size() */
  MW_WRANGE = 64,     /* status bit (warning): an operand's exponent spread exceeds the
                         spread the plan was made for; the error bound is not guaranteed */
  MW_EUNSUPPORTED = 128
};

/* forms of the product */
enum { MW_PLAIN = 0, MW_OZAKI = 1, MW_DOT = 2, MW_CRT = 3, MW_TEXTBOOK = 4 };

/* digit formats written by mw_split */
enum { MW_DIGITS_BF16 = 0, MW_DIGITS_F64 = 1 };
/* Operations of mw_elementwise (Table 1's add, mul and div). */
enum { MW_OP_ADD = 0, MW_OP_MUL = 1, MW_OP_DIV = 2 };

/* A plan fixes the slicing of a product.  mw_plan_gemm fills it from the error
 * analysis (see there); a caller may also set the fields directly.
 *   w      piece width in bits (MW_OZAKI: 7 or 8; MW_PLAIN: 1..26; MW_DOT: 24)
 *   S_A    pieces per entry of op(A); S_B pieces per entry of op(B)
 *   D      diagonals kept: pairs (p, q) with p < S_A, q < S_B, p + q < D
 *   group  diagonals fused into one 64-bit partial sum (MW_OZAKI)
 *   chunk  products of pieces accumulated in fp32 before a drain (MW_OZAKI;
 *          multiple of 64, chunk 2^(2w-2) <= 2^24)
 *   range_A, range_B  exponent spread (bits) the plan assumes for the rows of
 *          op(A) / columns of op(B); larger spreads raise MW_WRANGE.
 * MW_CRT reads the fields so: w = 1, S_A / S_B = fixed-point bits L_A / L_B of
 * the entries of op(A) / op(B) (T = sum_j trunc(x_j 2^(L - 2 - E))), D = number
 * of moduli (the first D of mw_crt_moduli), group = 1, chunk unused. */
typedef struct mw_plan {
  int m, mode, w, S_A, S_B, D, group, chunk, range_A, range_B;
} mw_plan;

/* Plan a product so that |C - C_exact| <= 2K 2^(-52m) (|op(A)||op(B)|)
 * componentwise for any operands whose rows of op(A) (columns of op(B)) span at
 * most range_A (range_B) binary orders of magnitude, measured as max minus min
 * of ilogb+1 over the nonzero entries.  Host only, no GPU work.
 * plan->w on input: 0 lets the planner choose (MW_OZAKI 8, MW_PLAIN the widest
 * width whose sums stay exact, MW_DOT 24); a width in range (2..8 for MW_OZAKI,
 * 4..26 for MW_PLAIN, 24 for MW_DOT) is used as given.  Zero the struct before
 * the call.  MW_DOT plans one inner product of length K (M = N = 1) with
 * S_A = S_B = the smallest compiled piece count that covers the analysis
 * (2: 4..8, 4: 8..12, 8: 17..21, 16: 35..36) and D <= S + 4.
 * MW_CRT takes L_A, L_B from the same truncation analysis (at bit
 * granularity) and the fewest moduli whose product P exceeds
 * 8 K 2^(L_A + L_B - 2) >= 8 max|X| (m = 2 or 4).
 * Returns MW_EINVAL for bad arguments, MW_EUNSUPPORTED if no plan fits the
 * exactness thresholds (e.g. K too long for MW_PLAIN, more bits than the
 * moduli of MW_CRT hold) or for m = 16 with MW_PLAIN.
 * Cites: Section 2 (the exactness threshold on the number of summed
 * products of pieces); the componentwise bound itself is the library's. */
int mw_plan_gemm(int m, int mode, int64_t M, int64_t N, int64_t K, int range_A, int range_B,
                 mw_plan *plan);

/* Steps 1-2 for one operand (Section 2; the quarters of the double double
 * inner product generalised to S pieces of w bits).
 * The logical operand has R rows (the output dimension) and K columns (the
 * reduction dimension).  trans = 0: X is stored R x K (X[r*ld + k]);
 * trans = 1: X is stored K x R (X[k*ld + r]).
 * Outputs (device memory owned by the caller):
 *   exps[r]   = E_r = max over the row of (ilogb(x_j) + 1) over nonzero words x_j,
 *               0 for an all-zero row;
 *   spread[r] = E_r - min over nonzero entries of (max_j ilogb(x_j) + 1);
 *   digits    S planes of R x digit_ld pieces, piece p of entry (r, k) at
 *             digits[(p * R + r) * digit_ld + k], as bfloat16 (format
 *             MW_DIGITS_BF16, w <= 9) or double (MW_DIGITS_F64); columns
 *             K..digit_ld-1 are written with zeros.  Piece p weighs
 *             2^(E_r + 2 - w (p + 1)); the pieces are the balanced base-2^w
 *             digits of T = sum_j trunc(x_j 2^(wS - 2 - E_r)).
 *   max_spread (may be NULL): one int updated with atomicMax of spread[r].
 * GPU-side errors: MW_ENONFINITE, MW_ERANGE (T outside [-2^(wS-1), 2^(wS-1))) in the status word;
 * MW_WRANGE when spread[r] > range (pass range < 0 to skip the check). */
int mw_split(int m, int trans, int64_t R, int64_t K, const double *X, int64_t ld,
             int64_t plane_stride, int w, int S, int format, void *digits, int64_t digit_ld,
             int32_t *exps, int32_t *spread, int32_t *max_spread, int range, mw_stream_t stream);

/* The residue form's moduli, in the order plans use them (a plan with D moduli
 * uses the first D): pairwise coprime, at most 513.  Copies min(n, total) of
 * them to moduli (may be NULL) and returns the total.  Host only.
 * Cites: Sections 1 and 4 (the Ozaki scheme the residue form follows); the
 * table itself is the library's. */
int mw_crt_moduli(int *moduli, int n);

/* Bytes of device workspace mw_gemm needs for this plan and shape.
 * No counterpart in the paper (device memory sizing). */
int mw_gemm_workspace_size(const mw_plan *plan, int64_t M, int64_t N, int64_t K, size_t *bytes);

/* Where mw_gemm keeps its intermediates inside ws, for inspection and tests:
 * offsets[0] int32 exponents and spreads: E_A[M], spread_A[M], E_B[N], spread_B[N],
 *            then the two largest spreads and two flags (MW_CRT: an operand's
 *            exponents were taken again over every word);
 * offsets[1] pieces of op(A): S_A planes of M x Kp (Kp = K rounded up to 64),
 *            bfloat16 (MW_OZAKI) or double (MW_PLAIN), layout as in mw_split;
 *            MW_CRT: D planes of balanced residues (bfloat16), plane i mod p_i;
 * offsets[2] pieces of op(B)^T: S_B planes of N x Kp (MW_CRT: D residue planes);
 * offsets[3] (MW_OZAKI) partial sums, one column-major plane per entry (entry
 *            (i, j) of a plane at j*M + i).  When min(S_A, S_B) * Kp * 2^(2w-2)
 *            < 2^31 every diagonal sum fits in 32 bits and the planes are the
 *            int32 s_t, t < D; otherwise int64 planes g < G holding
 *            V = sum_t s_t 2^(w (t1 - t)) over the diagonals of group g,
 *            [g*group, t1 = min(D, (g+1)*group) - 1].
 *            MW_CRT: D bfloat16 planes of M rows of N rounded up to 8 entries
 *            (row-major), plane i the balanced residue mod p_i of each entry's
 *            sum of products of residues.
 * bytes = total workspace size (same as mw_gemm_workspace_size).
 * No counterpart in the paper (device memory sizing). */
int mw_gemm_workspace_layout(const mw_plan *plan, int64_t M, int64_t N, int64_t K,
                             size_t offsets[4], size_t *bytes);

/* C = op(A) op(B), overwriting the m planes of C (M x N).  op(A) is M x K,
 * op(B) is K x N; transA/transB = 1 take the stored matrix transposed
 * (A stored K x M, B stored N x K).  plan->m words per entry in A, B and C.
 * ws: device workspace of at least mw_gemm_workspace_size() bytes; it holds the
 * pieces, the exponents and the diagonal partial sums; no memory is allocated.
 * Asynchronous on `stream`.  MW_CRT takes the shared exponents from the leading
 * words first and checks every entry while cutting it; an operand with an entry
 * whose later word is larger (input that is not normalised), not finite or out of
 * range is cut again with the exponents over every word.
 * Cites: Section 2 (error-free summation of pieces, the s_i) and
 * Section 4 (the matrix form, pieces of matrices on tensor cores; the Ozaki
 * scheme, whose residue form MW_CRT computes). */
int mw_gemm(const mw_plan *plan, int transA, int transB, int64_t M, int64_t N, int64_t K,
            const double *A, int64_t lda, int64_t plane_stride_a,
            const double *B, int64_t ldb, int64_t plane_stride_b,
            double *C, int64_t ldc, int64_t plane_stride_c,
            void *ws, size_t ws_bytes, mw_stream_t stream);

/* mw_gemm for callers that cannot allocate device memory.  The paper has no
 * counterpart; it exists for callers such as a plug-in inside a host program
 * that owns all device memory through its own pool (a framework's caching
 * allocator, a server with a fixed memory budget) and may not call cudaMalloc,
 * which synchronizes the device and takes memory the host does not account for.
 * Same arguments and result as mw_gemm without ws/ws_bytes: the workspace is a
 * fixed 32 MiB array that the library reserves on every device it is loaded on
 * and holds until the process exits; no memory is allocated or freed by the
 * call.  Products whose mw_gemm_workspace_size exceeds 32 MiB are rejected with
 * MW_ENOSPC (and a message) before any GPU work.  A call outside a stream
 * capture looks up the array's device address (cudaGetSymbolAddress) with the
 * device current; a call inside a capture uses the address the last call
 * outside one found on that device, so make a first call on every device
 * before any stream capture (MW_EINVAL otherwise).  Every call on a device
 * shares the array and leaves its contents behind (mw_gemm itself clears what
 * must start at zero); calls whose work overlaps on the GPU race on it, so
 * order them on one stream or otherwise serialise them. */
int mw_gemm_noalloc(const mw_plan *plan, int transA, int transB, int64_t M, int64_t N, int64_t K,
                    const double *A, int64_t lda, int64_t plane_stride_a,
                    const double *B, int64_t ldb, int64_t plane_stride_b,
                    double *C, int64_t ldc, int64_t plane_stride_c, mw_stream_t stream);

/* ---- inner products (Section 2: the s_i of an inner product; Table 2 times
 * 1,024 inner products of length 6,144) ------------------------------------ */

/* c_i = sum_k a_ik b_ik for i < count, every product error-free summed as in
 * Section 2 with the plan's pieces (mw_plan_gemm(m, MW_DOT, 1, 1, K, ...)):
 * |c_i - exact| <= 2K 2^(-52m) sum_k |a_ik||b_ik| for operands within the
 * plan's exponent spreads.  a_i is row i of A (count x K, m planes, row stride
 * lda, plane stride plane_stride_a), b_i row i of B (likewise); c_i is entry i
 * of every plane of C (plane stride plane_stride_c).  One CTA per inner product;
 * no workspace, asynchronous.  The shared exponent of a vector (ilogb + 1 of
 * its largest word) is found from the leading words and checked against every
 * word while cutting; a vector whose later word is larger (input that is not
 * normalised) is cut a second time.  MW_EINVAL for a plan of another form or bad
 * arguments, MW_EUNSUPPORTED for piece counts the kernel is not compiled for;
 * device status bits as for mw_gemm. */
int mw_dot_batched(const mw_plan *plan, int64_t count, int64_t K, const double *A, int64_t lda,
                   int64_t plane_stride_a, const double *B, int64_t ldb, int64_t plane_stride_b,
                   double *C, int64_t plane_stride_c, mw_stream_t stream);

/* Products of truncated power series with m-double coefficients (Section 1's
 * application; Section 2's diagonal sums s_i are these convolutions):
 *   c_si = sum_{k=0..i} a_sk b_s(i-k)   for every series s < count, i < n,
 * each coefficient the inner product of a_s0..a_si with b_si..b_s0, summed
 * error-free as in mw_dot_batched with the plan's pieces.  Plan it as one inner
 * product of length 1 (mw_plan_gemm(m, MW_DOT, 1, 1, 1, ...): the shortest
 * product needs the most bits), so that every coefficient meets
 * |c_si - exact| <= 2 (i+1) 2^(-52m) sum_k |a_sk| |b_s(i-k)|.  Series s of A is
 * row s (coefficient k at A[j * plane_stride_a + s * lda + k], word plane j),
 * likewise B; c_si goes to C[j * plane_stride_c + s * ldc + i].  One CTA per
 * coefficient; no workspace, asynchronous.  MW_EINVAL for bad arguments,
 * MW_EUNSUPPORTED for n beyond the kernel's int64 sums; device status bits as
 * for mw_dot_batched. */
int mw_convolve_batched(const mw_plan *plan, int64_t count, int64_t n, const double *A,
                        int64_t lda, int64_t plane_stride_a, const double *B, int64_t ldb,
                        int64_t plane_stride_b, double *C, int64_t ldc, int64_t plane_stride_c,
                        mw_stream_t stream);

/* Entry-by-entry m-double arithmetic (Table 1: the m-double addition,
 * multiplication and division whose costs in doubles the paper counts):
 *   C_e = A_e op B_e,  e < n,  op = MW_OP_ADD, MW_OP_MUL or MW_OP_DIV,
 * with MW_TEXTBOOK's operations (two_sum, two_prod, renormalisation into m
 * words); division is long division (m + 1 quotient words from the leading word
 * of the remainder, the remainder reduced by each word times B, renormalised),
 * within 2^(1-52m) |A_e / B_e| of the exact quotient on the tested inputs.
 * Entry e of word plane j of A at A[j * plane_stride_a + e] (likewise B, C);
 * plane strides at least n; C may be A or B (each entry is read before it is
 * written).  m = 2, 4 or 8.  One thread per entry; no workspace,
 * asynchronous on `stream`; nothing is checked on the device (a zero leading
 * word of B gives IEEE infinities or NaNs).  MW_EINVAL for a bad op, m, n,
 * stride or NULL pointer (n = 0 does nothing). */
int mw_elementwise(int op, int m, int64_t n, const double *A, int64_t plane_stride_a,
                   const double *B, int64_t plane_stride_b, double *C, int64_t plane_stride_c,
                   mw_stream_t stream);

/* ---- batches of independent products (power-series coefficient convolutions,
 * Section 1, come as many small products of uneven sizes) -------------------- */

/* One product of a batch: C = A B, A M x K, B K x N, C M x N, every matrix m
 * planes of row-major doubles in device memory (no transposes). */
typedef struct mw_problem {
  int64_t M, N, K;
  const double *A;
  int64_t lda, plane_stride_a;
  const double *B;
  int64_t ldb, plane_stride_b;
  double *C;
  int64_t ldc, plane_stride_c;
} mw_problem;

/* Host-side summary of a batch (sizes only); mw_batch_describe fills it. */
typedef struct mw_batch {
  int count;
  int64_t sum_M, sum_N, sum_MN, max_M, max_N, min_K, max_K;
} mw_batch;

/* shapes: host array of count x {M, N, K}. Host only.
 * No counterpart in the paper (batch bookkeeping). */
int mw_batch_describe(int count, const int64_t *shapes, mw_batch *batch);

/* Bytes of device workspace for mw_gemm_batched with this plan (MW_OZAKI).
 * No counterpart in the paper (device memory sizing). */
int mw_gemm_batched_workspace_size(const mw_plan *plan, const mw_batch *batch, size_t *bytes);

/* Bytes of device workspace mw_measure_spread_batched needs for this batch
 * (host only; at most 8192 + 256 count + 16 (sum_M + sum_N) + sum_MN / 32).
 * MW_EINVAL for m outside {2, 4, 8, 16} or a bad batch summary.
 * No counterpart in the paper (device memory sizing). */
int mw_measure_spread_batched_workspace_size(int m, const mw_batch *batch, size_t *bytes);

/* Exponent spreads over all rows of the A_i and all columns of the B_i
 * (synchronizes); input to mw_plan_gemm for the batch.  ws: device workspace
 * of at least mw_measure_spread_batched_workspace_size bytes (MW_ENOSPC
 * otherwise).
 * Cites: Section 2 (the shared-exponent assumption the spreads measure). */
int mw_measure_spread_batched(int m, const mw_batch *batch, const mw_problem *problems,
                              void *ws, size_t ws_bytes, int *range_A, int *range_B,
                              mw_stream_t stream);

/* C_i = A_i B_i for every problem of the batch in the Ozaki form (m = 2, 4, 8
 * or 16), one plan for all (plan it with the smallest K of the batch for the
 * error bound; its group
 * must also fit the largest K).  problems: device array of batch->count
 * descriptors.  Launches a short prologue (offsets of every problem's pieces
 * and partial sums, computed on the GPU from the descriptors), one split of all
 * operands, one persistent product kernel over (problem, tile, diagonal group)
 * work items, one fusion; no host synchronisation, so the call can be captured
 * in a CUDA graph and replayed while the descriptors and ws keep their
 * addresses.  For load balance order the problems by decreasing size.
 * Cites: Section 4 (matrix products of pieces); Section 1 (the power series
 * that need many small products) motivates the batch. */
int mw_gemm_batched(const mw_plan *plan, const mw_batch *batch, const mw_problem *problems,
                    void *ws, size_t ws_bytes, mw_stream_t stream);

/* Exponent spreads (max over rows of op(A), columns of op(B)) measured on the
 * GPU; synchronizes the stream.  ws as for mw_gemm with any plan of this m
 * (only 2 * (M + N + 1) int32 are used).  Feed the results to mw_plan_gemm.
 * Cites: Section 2 (the shared-exponent assumption the spreads measure). */
int mw_measure_spread(int m, int transA, int transB, int64_t M, int64_t N, int64_t K,
                      const double *A, int64_t lda, int64_t plane_stride_a,
                      const double *B, int64_t ldb, int64_t plane_stride_b,
                      void *ws, size_t ws_bytes, int *range_A, int *range_B, mw_stream_t stream);

/* Adjoint of C = A B for a loss L with dL/dC = G (M x N), all m-doubles:
 * dA = G B^T (M x K) and dB = A^T G (K x N), each computed like mw_gemm with
 * the transposes folded into the slicing.  plan_dA and plan_dB are plans of the
 * two products (shapes M x K x N and K x N x M).  ws: at least the larger of
 * their workspace sizes.  Either output may be NULL to skip it.
 * No counterpart in the paper (the adjoint); its two products are
 * computed as mw_gemm computes C (Sections 2 and 4). */
int mw_gemm_backward(const mw_plan *plan_dA, const mw_plan *plan_dB,
                     int64_t M, int64_t N, int64_t K,
                     const double *A, int64_t lda, int64_t plane_stride_a,
                     const double *B, int64_t ldb, int64_t plane_stride_b,
                     const double *G, int64_t ldg, int64_t plane_stride_g,
                     double *dA, int64_t ldda, int64_t plane_stride_da,
                     double *dB, int64_t lddb, int64_t plane_stride_db,
                     void *ws, size_t ws_bytes, mw_stream_t stream);

/* Profiling hook: while set, every mw_gemm and mw_gemm_batched records
 * events[0] on its stream before the first launch, events[1] after the pieces
 * are cut (before the product kernel), events[2] after the product kernel and
 * events[3] after the last launch.  events are cudaEvent_t created by the caller; pass NULL (or
 * n = 0) to stop.  Process-wide setting, not thread safe.
 * No counterpart in the paper (profiling). */
int mw_set_phase_events(void *const *events, int n);

/* Read the device status word of the current device (synchronizes the device);
 * clear != 0 resets it to zero afterwards.
 * No counterpart in the paper (error reporting). */
int mw_get_status(int *bits, int clear);

/* Message for the last host-side error of the calling thread ("" if none). */
const char *mw_last_error(void);

/* Diagnostic with no counterpart in the paper: one CTA waits on a shared-memory
 * barrier that nothing completes, with the bounded wait the pipeline kernels
 * use but a limit of limit_us microseconds (1 .. 10^7); the wait gives up,
 * raises MW_ETIMEOUT in the status word and the kernel returns, leaving the
 * context usable.  Asynchronous on `stream`; read the bit with mw_get_status. */
int mw_selftest_timeout(unsigned int limit_us, mw_stream_t stream);

/* Library version string. */
const char *mw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MW_H */
