/* Textbook ("ordinary") m-double matrix product on the CPU: oracle part O1.
 *
 * Test infrastructure only: the tests, the smoke check and the benchmark's CPU
 * baseline call it; the GPU library never does.
 *
 * Table 2 of the paper compares its vectorized inner products with "ordinary"
 * ones in which every term a_k * b_k is an m-double multiplication followed by
 * an m-double addition.  This file is that ordinary product for a matrix,
 * C_ij = sum_k a_ik * b_kj, built from the error-free transformations of
 * floating-point arithmetic:
 *   two_sum      (Knuth):  s = fl(a+b), e = a + b - s exactly, 6 flops;
 *   fast_two_sum (Dekker): the same when |a| >= |b|, 3 flops;
 *   split        (Veltkamp/Dekker, factor 2^27+1): a = hi + lo, 4 flops;
 *   two_prod     (Dekker, no fused multiply-add): p + e = a*b exactly, 17 flops.
 * m = 2 uses the classic double-double add (two two_sums, two fast_two_sums,
 * 20 flops, Table 1) and multiply (two_prod plus cross terms, 24 flops).
 * m = 4, 8 and 16 form the exact partial products of each magnitude level
 * (i + j = l) with two_prod, keep the rounded products of level m, and
 * renormalise the level-ordered terms into m words by repeated bottom-up
 * two_sum sweeps, each sweep peeling off one word.  Division (md_div) is long
 * division with m + 1 quotient words built from these operations.
 *
 * Must be compiled with -ffp-contract=off so that no multiply-add is fused.
 * Layout: every matrix is m planes of row-major doubles, plane j at j*rows*cols.
 */
#include <stdint.h>
#include <string.h>

#define MAXM 16
#define MAXT 320

static inline double two_sum(double a, double b, double *e) {
  double s = a + b;
  double bv = s - a;
  double av = s - bv;
  *e = (a - av) + (b - bv);
  return s;
}

static inline double fast_two_sum(double a, double b, double *e) {
  double s = a + b;
  *e = b - (s - a);
  return s;
}

static inline void split(double a, double *hi, double *lo) {
  double c = 134217729.0 * a;
  *hi = c - (c - a);
  *lo = a - *hi;
}

static inline double two_prod(double a, double b, double *e) {
  double p = a * b, ah, al, bh, bl;
  split(a, &ah, &al);
  split(b, &bh, &bl);
  *e = ((ah * bh - p) + ah * bl + al * bh) + al * bl;
  return p;
}

static inline void dd_add(const double *a, const double *b, double *r) {
  double s, e, t, f;
  s = two_sum(a[0], b[0], &e);
  t = two_sum(a[1], b[1], &f);
  e += t;
  s = fast_two_sum(s, e, &e);
  e += f;
  s = fast_two_sum(s, e, &e);
  r[0] = s;
  r[1] = e;
}

static inline void dd_mul(const double *a, const double *b, double *r) {
  double p, e;
  p = two_prod(a[0], b[0], &e);
  e += a[0] * b[1] + a[1] * b[0];
  p = fast_two_sum(p, e, &e);
  r[0] = p;
  r[1] = e;
}

/* Renormalise n level-ordered terms into m words: each pass sums the terms
 * bottom-up with two_sum, keeps the top sum as the next word and the exact
 * rounding errors as the terms of the next pass. */
static void renorm(double *x, int n, int m, double *r) {
  for (int j = 0; j < m; ++j) {
    if (n <= 0) { r[j] = 0.0; continue; }
    double s = x[n - 1];
    for (int i = n - 2; i >= 0; --i) {
      double e;
      s = two_sum(x[i], s, &e);
      x[i + 1] = e;
    }
    r[j] = s;
    /* terms of the next pass: x[1..n-1]; drop exact zeros */
    int k = 0;
    for (int i = 1; i < n; ++i)
      if (x[i] != 0.0) x[k++] = x[i];
    n = k;
  }
}

static void md_add(int m, const double *a, const double *b, double *r) {
  if (m == 2) { dd_add(a, b, r); return; }
  double t[2 * MAXM];
  for (int i = 0; i < m; ++i) { t[2 * i] = a[i]; t[2 * i + 1] = b[i]; }
  renorm(t, 2 * m, m, r);
}

static void md_mul(int m, const double *a, const double *b, double *r) {
  if (m == 2) { dd_mul(a, b, r); return; }
  /* level l holds the high parts of a_i b_j with i+j = l and the low parts
   * of the level l-1 products; level m holds rounded a_i b_j with i+j = m. */
  double lo_prev[MAXM + 1];
  int nlo_prev = 0;
  double t[MAXT];
  int n = 0;
  for (int l = 0; l < m; ++l) {
    double lo_cur[MAXM + 1];
    int nlo_cur = 0;
    for (int i = 0; i <= l; ++i) {
      double e;
      t[n++] = two_prod(a[i], b[l - i], &e);
      lo_cur[nlo_cur++] = e;
    }
    for (int i = 0; i < nlo_prev; ++i) t[n++] = lo_prev[i];
    for (int i = 0; i < nlo_cur; ++i) lo_prev[i] = lo_cur[i];
    nlo_prev = nlo_cur;
  }
  for (int i = 1; i < m; ++i) t[n++] = a[i] * b[m - i];
  for (int i = 0; i < nlo_prev; ++i) t[n++] = lo_prev[i];
  renorm(t, n, m, r);
}

/* m-double division a / b by long division (Table 1's div; the paper gives only
 * its operation count, so the algorithm is this file's): m + 1 quotient words,
 * q_i = fl(r_0 / b_0) from the leading word of the remainder r (r = a at
 * first), r = r - q_i b after each of the first m (q_i b an m-double product of
 * (q_i, 0, ..., 0) and b, subtracted as an m-double addition of its negation,
 * for m >= 4 renormalised once more), then the m + 1 quotient words renormalised
 * into m. */
static void md_div(int m, const double *a, const double *b, double *r) {
  double rem[MAXM], q[MAXM + 1], qv[MAXM], t[MAXM], s[MAXM];
  memcpy(rem, a, sizeof(double) * m);
  for (int i = 0; i <= m; ++i) {
    q[i] = rem[0] / b[0];
    if (i == m) break;
    memset(qv, 0, sizeof(double) * m);
    qv[0] = q[i];
    md_mul(m, qv, b, t);
    for (int w = 0; w < m; ++w) t[w] = -t[w];
    md_add(m, rem, t, s);
    /* the sum cancels in its leading words: for m >= 4 renormalise it once more,
     * so that its leading word, which gives the next quotient word, leads */
    if (m > 2) renorm(s, m, m, rem);
    else memcpy(rem, s, sizeof(double) * m);
  }
  renorm(q, m + 1, m, r);
}

/* C rows listed in `rows` (nrows of them), all N columns:
 * C[j][rows[r]][c] = sum_k A[.][rows[r]][k] * B[.][k][c] in m-double arithmetic.
 * Rows are distributed over `nthreads` OpenMP threads. */
void tb_gemm_rows(int m, int64_t M, int64_t N, int64_t K, const double *A, const double *B,
                  double *C, const int64_t *rows, int64_t nrows, int nthreads) {
  const int64_t pa = M * K, pb = K * N, pc = M * N;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int64_t r = 0; r < nrows; ++r) {
    const int64_t i = rows[r];
    for (int64_t c = 0; c < N; ++c) {
      double acc[MAXM] = {0}, a[MAXM], b[MAXM], p[MAXM], s[MAXM];
      for (int64_t k = 0; k < K; ++k) {
        for (int w = 0; w < m; ++w) {
          a[w] = A[w * pa + i * K + k];
          b[w] = B[w * pb + k * N + c];
        }
        md_mul(m, a, b, p);
        md_add(m, acc, p, s);
        memcpy(acc, s, sizeof(double) * m);
      }
      for (int w = 0; w < m; ++w) C[w * pc + i * N + c] = acc[w];
    }
  }
}

/* Single operations, for tests against the Python twin. */
void tb_mul(int m, const double *a, const double *b, double *r) { md_mul(m, a, b, r); }
void tb_add(int m, const double *a, const double *b, double *r) { md_add(m, a, b, r); }
void tb_div(int m, const double *a, const double *b, double *r) { md_div(m, a, b, r); }

/* Elementwise over n entries, m planes each (plane j of x at x + j*n):
 * op 0 add, 1 mul, 2 div; entries distributed over `nthreads` OpenMP threads. */
void tb_elementwise(int op, int m, int64_t n, const double *A, const double *B, double *C,
                    int nthreads) {
#pragma omp parallel for schedule(static) num_threads(nthreads)
  for (int64_t e = 0; e < n; ++e) {
    double a[MAXM], b[MAXM], r[MAXM];
    for (int w = 0; w < m; ++w) {
      a[w] = A[w * n + e];
      b[w] = B[w * n + e];
    }
    if (op == 0) md_add(m, a, b, r);
    else if (op == 1) md_mul(m, a, b, r);
    else md_div(m, a, b, r);
    for (int w = 0; w < m; ++w) C[w * n + e] = r[w];
  }
}

int tb_max_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
