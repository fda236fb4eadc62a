/*
 * Plain CPU oracle for Randomly Pivoted LU (RPLU).  TEST INFRASTRUCTURE ONLY:
 * it is called from tests/, from __graft_entry__.smoke() and from the
 * cpu_baseline leg of bench.py, never from the product path.  It shares no code
 * with the CUDA library.
 *
 * It is slow and sequential on purpose: every loop runs in index order, every
 * sum is a left-to-right FP64 (or complex128) sum, and the file is compiled
 * with -ffp-contract=off so that no multiply-add is fused.
 *
 * What it computes (paper: Gilles & Wilber, "Low-Rank Approximation by
 * Randomly Pivoted LU"):
 *   - rplu dense form: Algorithm 1 (Sec. 1) -- at step t the pivot (i, j) is
 *     drawn with probability |S_ij|^2 / ||S||_F^2 (Sec. 1, pivot law), by the
 *     two-stage rule of Sec. 4.1 (row by squared row norm, then column by the
 *     squared entries of that row); L(:,t) = S(:,j)/S_ij, U(t,:) = S(i,:),
 *     S <- S - L(:,t) U(t,:) (Eq. residual_update).  Row norms are recomputed
 *     from S after each step.
 *   - rplu matrix-free Cauchy form: the same iteration with A_ij = 1/(x_i - y_j)
 *     generated on demand (Sec. 5.1, p = 1, G = B = 1), residual rows and
 *     columns formed as A(i,:) - L(i,:)U and A(:,j) - L U(:,j) (the LU-form
 *     analogue of Algorithm 2, Sec. 4.1), and the squared row norms updated
 *     by the formula of Sec. 4.1 "Row norm updates".
 *
 * Readings where the paper is silent (all shared with the CUDA path as a
 * specification, not as code):
 *   - draws: U01(seed, t, s, a) from the SplitMix64 output function (Steele,
 *     Lea & Flood 2014) evaluated at seed + gamma*(1 + 128 t + 2 a + s), t the
 *     step, s = 0 for the row draw and 1 for the column draw, a the redraw
 *     attempt (< 64);
 *   - inverse CDF: the smallest index with prefix sum > u * total; when
 *     rounding leaves none, the last index with positive weight;
 *   - columns already pivoted get weight 0 in the column draw; pivoted rows
 *     and columns of S are set to exactly 0;
 *   - L(i_t, t) := 1 and L(I_prev, t) := 0, U(t, J_prev) := 0;
 *   - a sampled row whose masked weights sum to 0 gets d_i := 0 and the row is
 *     drawn again (attempt + 1), at most 64 attempts;
 *   - stop when the total is 0 or total <= tol^2 * initial total (tol > 0);
 *   - C2 mode (complete 2-norm pivoting, Sec. 2): argmax of d, then argmax of
 *     the row's squared entries; COMPLETE mode: argmax |S_pq| over all
 *     entries (Sec. 1); ties go to the smallest (row-major) index.
 *
 * Parity pins for every function are listed in tests/test_oracle_*.py.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MODE_RANDOM 0
#define MODE_C2 1
#define MODE_COMPLETE 2
#define MODE_GIVEN 3

#define MAX_ATTEMPTS 64

typedef double complex cplx;

/* ------------------------------------------------------------------ draws */

static uint64_t splitmix64_output(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double oracle_u01(uint64_t seed, int64_t t, int32_t s, int32_t a) {
  const uint64_t gamma = 0x9E3779B97F4A7C15ULL;
  uint64_t counter = 1u + 128u * (uint64_t)t + 2u * (uint64_t)a + (uint64_t)s;
  uint64_t z = splitmix64_output(seed + gamma * counter);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0); /* 2^-53 */
}

/* --------------------------------------------------------------- sampling */

/* Smallest index i with (w_0 + ... + w_i) > target, sums in index order.  If
 * none exists, the last index with w_i > 0 (or -1 if all are zero).  *margin
 * receives the distance from target to the nearer boundary of the chosen cell,
 * divided by total (how close the draw came to selecting a neighbour). */
int64_t oracle_inverse_cdf(const double* w, int64_t n, double target, double total, double* margin) {
  double c = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double lo = c;
    c = c + w[i];
    if (c > target) {
      double dlo = target - lo, dhi = c - target;
      if (margin) *margin = (dlo < dhi ? dlo : dhi) / total;
      return i;
    }
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    if (w[i] > 0.0) {
      if (margin) *margin = 0.0;
      return i;
    }
  }
  if (margin) *margin = 0.0;
  return -1;
}

static int64_t argmax_first(const double* w, int64_t n) {
  int64_t best = -1;
  double bv = -1.0;
  for (int64_t i = 0; i < n; ++i)
    if (w[i] > bv) { bv = w[i]; best = i; }
  return best;
}

static double sum_in_order(const double* w, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s = s + w[i];
  return s;
}

static double abs2(cplx z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

/* ------------------------------------------------- dense form, real FP64 */

/* A: n x m row-major (lda = m).  Outputs: piv_I[k], piv_J[k]; L n x k column-major;
 * U k x m row-major; T_hist[k+1] = ||S^(t)||_F^2 before step t and after the
 * last step; row_margin[k], col_margin[k]; *k_done.  Returns 0, or -1 on an
 * invalid argument / allocation failure. */
int oracle_rplu_dense_f64(const double* A, int64_t n, int64_t m, int64_t k, uint64_t seed, int32_t mode,
                          const int64_t* given_I, const int64_t* given_J, double tol, int64_t* piv_I, int64_t* piv_J,
                          double* L, double* U, double* T_hist, double* row_margin, double* col_margin,
                          int64_t* k_done) {
  if (n < 0 || m < 0 || k < 0 || k > (n < m ? n : m)) return -1;
  double* S = (double*)malloc(sizeof(double) * (size_t)(n * m > 0 ? n * m : 1));
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  char* col_used = (char*)calloc((size_t)(m > 0 ? m : 1), 1);
  char* row_used = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!S || !d || !w || !col_used || !row_used) { free(S); free(d); free(w); free(col_used); free(row_used); return -1; }
  memcpy(S, A, sizeof(double) * (size_t)(n * m));
  memset(L, 0, sizeof(double) * (size_t)(n * k));
  memset(U, 0, sizeof(double) * (size_t)(k * m));
  for (int64_t p = 0; p < n; ++p) {
    double s = 0.0;
    for (int64_t q = 0; q < m; ++q) s = s + S[p * m + q] * S[p * m + q];
    d[p] = s;
  }
  double T0 = sum_in_order(d, n);
  int64_t t = 0;
  for (; t < k; ++t) {
    double T = sum_in_order(d, n);
    T_hist[t] = T;
    if (!(T > 0.0) || (tol > 0.0 && T <= tol * tol * T0)) break;
    int64_t i = -1, j = -1;
    double rm = 0.0, cm = 0.0;
    int ok = 0;
    for (int attempt = 0; attempt < MAX_ATTEMPTS && !ok; ++attempt) {
      if (mode == MODE_GIVEN) {
        i = given_I[t];
        j = given_J[t];
        ok = 1;
        break;
      }
      if (mode == MODE_COMPLETE) {
        double best = -1.0;
        for (int64_t p = 0; p < n; ++p)
          for (int64_t q = 0; q < m; ++q) {
            double v = S[p * m + q] * S[p * m + q];
            if (v > best) { best = v; i = p; j = q; }
          }
        ok = 1;
        break;
      }
      if (mode == MODE_RANDOM) {
        double u1 = oracle_u01(seed, t, 0, attempt);
        i = oracle_inverse_cdf(d, n, u1 * T, T, &rm);
      } else { /* MODE_C2 */
        i = argmax_first(d, n);
      }
      for (int64_t q = 0; q < m; ++q) w[q] = col_used[q] ? 0.0 : S[i * m + q] * S[i * m + q];
      double R = sum_in_order(w, m);
      if (!(R > 0.0)) {
        d[i] = 0.0;
        T = sum_in_order(d, n);
        if (!(T > 0.0)) break;
        continue;
      }
      if (mode == MODE_RANDOM) {
        double u2 = oracle_u01(seed, t, 1, attempt);
        j = oracle_inverse_cdf(w, m, u2 * R, R, &cm);
      } else {
        j = argmax_first(w, m);
      }
      ok = 1;
    }
    if (!ok) break;
    double a = S[i * m + j];
    for (int64_t q = 0; q < m; ++q) U[t * m + q] = col_used[q] ? 0.0 : S[i * m + q];
    for (int64_t p = 0; p < n; ++p) L[t * n + p] = row_used[p] ? 0.0 : S[p * m + j] / a;
    L[t * n + i] = 1.0;
    piv_I[t] = i;
    piv_J[t] = j;
    if (row_margin) row_margin[t] = rm;
    if (col_margin) col_margin[t] = cm;
    row_used[i] = 1;
    col_used[j] = 1;
    for (int64_t p = 0; p < n; ++p)
      for (int64_t q = 0; q < m; ++q) S[p * m + q] = S[p * m + q] - L[t * n + p] * U[t * m + q];
    for (int64_t q = 0; q < m; ++q) S[i * m + q] = 0.0;
    for (int64_t p = 0; p < n; ++p) S[p * m + j] = 0.0;
    for (int64_t p = 0; p < n; ++p) {
      double s = 0.0;
      for (int64_t q = 0; q < m; ++q) s = s + S[p * m + q] * S[p * m + q];
      d[p] = s;
    }
  }
  *k_done = t;
  T_hist[t] = sum_in_order(d, n);
  free(S); free(d); free(w); free(col_used); free(row_used);
  return 0;
}

/* -------------------------------------------- dense form, complex128 */

int oracle_rplu_dense_c128(const cplx* A, int64_t n, int64_t m, int64_t k, uint64_t seed, int32_t mode,
                           const int64_t* given_I, const int64_t* given_J, double tol, int64_t* piv_I, int64_t* piv_J,
                           cplx* L, cplx* U, double* T_hist, double* row_margin, double* col_margin,
                           int64_t* k_done) {
  if (n < 0 || m < 0 || k < 0 || k > (n < m ? n : m)) return -1;
  cplx* S = (cplx*)malloc(sizeof(cplx) * (size_t)(n * m > 0 ? n * m : 1));
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  char* col_used = (char*)calloc((size_t)(m > 0 ? m : 1), 1);
  char* row_used = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!S || !d || !w || !col_used || !row_used) { free(S); free(d); free(w); free(col_used); free(row_used); return -1; }
  memcpy(S, A, sizeof(cplx) * (size_t)(n * m));
  memset(L, 0, sizeof(cplx) * (size_t)(n * k));
  memset(U, 0, sizeof(cplx) * (size_t)(k * m));
  for (int64_t p = 0; p < n; ++p) {
    double s = 0.0;
    for (int64_t q = 0; q < m; ++q) s = s + abs2(S[p * m + q]);
    d[p] = s;
  }
  double T0 = sum_in_order(d, n);
  int64_t t = 0;
  for (; t < k; ++t) {
    double T = sum_in_order(d, n);
    T_hist[t] = T;
    if (!(T > 0.0) || (tol > 0.0 && T <= tol * tol * T0)) break;
    int64_t i = -1, j = -1;
    double rm = 0.0, cm = 0.0;
    int ok = 0;
    for (int attempt = 0; attempt < MAX_ATTEMPTS && !ok; ++attempt) {
      if (mode == MODE_GIVEN) {
        i = given_I[t];
        j = given_J[t];
        ok = 1;
        break;
      }
      if (mode == MODE_COMPLETE) {
        double best = -1.0;
        for (int64_t p = 0; p < n; ++p)
          for (int64_t q = 0; q < m; ++q) {
            double v = abs2(S[p * m + q]);
            if (v > best) { best = v; i = p; j = q; }
          }
        ok = 1;
        break;
      }
      if (mode == MODE_RANDOM) {
        double u1 = oracle_u01(seed, t, 0, attempt);
        i = oracle_inverse_cdf(d, n, u1 * T, T, &rm);
      } else {
        i = argmax_first(d, n);
      }
      for (int64_t q = 0; q < m; ++q) w[q] = col_used[q] ? 0.0 : abs2(S[i * m + q]);
      double R = sum_in_order(w, m);
      if (!(R > 0.0)) {
        d[i] = 0.0;
        T = sum_in_order(d, n);
        if (!(T > 0.0)) break;
        continue;
      }
      if (mode == MODE_RANDOM) {
        double u2 = oracle_u01(seed, t, 1, attempt);
        j = oracle_inverse_cdf(w, m, u2 * R, R, &cm);
      } else {
        j = argmax_first(w, m);
      }
      ok = 1;
    }
    if (!ok) break;
    cplx a = S[i * m + j];
    for (int64_t q = 0; q < m; ++q) U[t * m + q] = col_used[q] ? 0.0 : S[i * m + q];
    for (int64_t p = 0; p < n; ++p) L[t * n + p] = row_used[p] ? 0.0 : S[p * m + j] / a;
    L[t * n + i] = 1.0;
    piv_I[t] = i;
    piv_J[t] = j;
    if (row_margin) row_margin[t] = rm;
    if (col_margin) col_margin[t] = cm;
    row_used[i] = 1;
    col_used[j] = 1;
    for (int64_t p = 0; p < n; ++p)
      for (int64_t q = 0; q < m; ++q) S[p * m + q] = S[p * m + q] - L[t * n + p] * U[t * m + q];
    for (int64_t q = 0; q < m; ++q) S[i * m + q] = 0.0;
    for (int64_t p = 0; p < n; ++p) S[p * m + j] = 0.0;
    for (int64_t p = 0; p < n; ++p) {
      double s = 0.0;
      for (int64_t q = 0; q < m; ++q) s = s + abs2(S[p * m + q]);
      d[p] = s;
    }
  }
  *k_done = t;
  T_hist[t] = sum_in_order(d, n);
  free(S); free(d); free(w); free(col_used); free(row_used);
  return 0;
}

/* ------------------------------------------ matrix-free Cauchy form */

static cplx cauchy_entry(const cplx* x, const cplx* y, int64_t p, int64_t q) { return 1.0 / (x[p] - y[q]); }

/* x (n), y (m) complex points; A_pq = 1/(x_p - y_q) is never stored.  Outputs
 * as in the dense form, plus d_out[n], the row-norm estimates after the last
 * step.  Modes: RANDOM, C2, GIVEN.  Returns 0 or -1. */
int oracle_rplu_cauchy(const cplx* x, const cplx* y, int64_t n, int64_t m, int64_t k, uint64_t seed, int32_t mode,
                       const int64_t* given_I, const int64_t* given_J, double tol, int64_t* piv_I, int64_t* piv_J, cplx* L,
                       cplx* U, double* d_out, double* T_hist, double* row_margin, double* col_margin,
                       int64_t* k_done) {
  if (n < 0 || m < 0 || k < 0 || k > (n < m ? n : m) || mode == MODE_COMPLETE) return -1;
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* wcol = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  cplx* r = (cplx*)malloc(sizeof(cplx) * (size_t)(m > 0 ? m : 1));
  cplx* c = (cplx*)malloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1));
  cplx* g = (cplx*)malloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1));
  cplx* v = (cplx*)malloc(sizeof(cplx) * (size_t)(k > 0 ? k : 1));
  char* col_used = (char*)calloc((size_t)(m > 0 ? m : 1), 1);
  char* row_used = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!d || !wcol || !r || !c || !g || !v || !col_used || !row_used) {
    free(d); free(wcol); free(r); free(c); free(g); free(v); free(col_used); free(row_used);
    return -1;
  }
  memset(L, 0, sizeof(cplx) * (size_t)(n * k));
  memset(U, 0, sizeof(cplx) * (size_t)(k * m));
  /* initial squared row norms d_p = sum_q |A_pq|^2 */
  for (int64_t p = 0; p < n; ++p) {
    double s = 0.0;
    for (int64_t q = 0; q < m; ++q) s = s + abs2(cauchy_entry(x, y, p, q));
    d[p] = s;
  }
  double T0 = sum_in_order(d, n);
  int64_t t = 0;
  for (; t < k; ++t) {
    double T = sum_in_order(d, n);
    T_hist[t] = T;
    if (!(T > 0.0) || (tol > 0.0 && T <= tol * tol * T0)) break;
    int64_t i = -1, j = -1;
    double rm = 0.0, cm = 0.0;
    int ok = 0;
    for (int attempt = 0; attempt < MAX_ATTEMPTS && !ok; ++attempt) {
      if (mode == MODE_GIVEN) i = given_I[t];
      else if (mode == MODE_RANDOM) {
        double u1 = oracle_u01(seed, t, 0, attempt);
        i = oracle_inverse_cdf(d, n, u1 * T, T, &rm);
      } else i = argmax_first(d, n);
      /* residual row r = A(i,:) - L(i,0:t) U(0:t,:) */
      for (int64_t q = 0; q < m; ++q) {
        cplx s = cauchy_entry(x, y, i, q);
        for (int64_t s_ = 0; s_ < t; ++s_) s = s - L[s_ * n + i] * U[s_ * m + q];
        r[q] = s;
      }
      if (mode == MODE_GIVEN) { j = given_J[t]; ok = 1; break; }
      for (int64_t q = 0; q < m; ++q) wcol[q] = col_used[q] ? 0.0 : abs2(r[q]);
      double R = sum_in_order(wcol, m);
      if (!(R > 0.0)) {
        d[i] = 0.0;
        T = sum_in_order(d, n);
        if (!(T > 0.0)) break;
        continue;
      }
      if (mode == MODE_RANDOM) {
        double u2 = oracle_u01(seed, t, 1, attempt);
        j = oracle_inverse_cdf(wcol, m, u2 * R, R, &cm);
      } else j = argmax_first(wcol, m);
      ok = 1;
    }
    if (!ok) break;
    cplx a = r[j];
    /* residual column c = A(:,j) - L(:,0:t) U(0:t,j) */
    for (int64_t p = 0; p < n; ++p) {
      cplx s = cauchy_entry(x, y, p, j);
      for (int64_t s_ = 0; s_ < t; ++s_) s = s - L[s_ * n + p] * U[s_ * m + j];
      c[p] = s;
    }
    for (int64_t q = 0; q < m; ++q) U[t * m + q] = col_used[q] ? 0.0 : r[q];
    for (int64_t p = 0; p < n; ++p) L[t * n + p] = row_used[p] ? 0.0 : c[p] / a;
    L[t * n + i] = 1.0;
    piv_I[t] = i;
    piv_J[t] = j;
    if (row_margin) row_margin[t] = rm;
    if (col_margin) col_margin[t] = cm;
    row_used[i] = 1;
    col_used[j] = 1;
    /* g = S^(t) conj(u),  u = U(t,:),  S^(t) = A - L(:,0:t) U(0:t,:) */
    double unorm2 = 0.0;
    for (int64_t q = 0; q < m; ++q) unorm2 = unorm2 + abs2(U[t * m + q]);
    for (int64_t s_ = 0; s_ < t; ++s_) {
      cplx s = 0.0;
      for (int64_t q = 0; q < m; ++q) s = s + U[s_ * m + q] * conj(U[t * m + q]);
      v[s_] = s;
    }
    for (int64_t p = 0; p < n; ++p) {
      cplx s = 0.0;
      for (int64_t q = 0; q < m; ++q) s = s + cauchy_entry(x, y, p, q) * conj(U[t * m + q]);
      for (int64_t s_ = 0; s_ < t; ++s_) s = s - L[s_ * n + p] * v[s_];
      g[p] = s;
    }
    /* d_p <- d_p - 2 Re(conj(l_p) g_p) + |l_p|^2 ||u||^2  (Sec. 4.1 row norm update) */
    for (int64_t p = 0; p < n; ++p) {
      cplx l = L[t * n + p];
      double nv = d[p] - 2.0 * creal(conj(l) * g[p]) + abs2(l) * unorm2;
      d[p] = nv > 0.0 ? nv : 0.0;
    }
    d[i] = 0.0;
  }
  *k_done = t;
  T_hist[t] = sum_in_order(d, n);
  if (d_out) memcpy(d_out, d, sizeof(double) * (size_t)n);
  free(d); free(wcol); free(r); free(c); free(g); free(v); free(col_used); free(row_used);
  return 0;
}

/* -------------------------------------------- Cauchy-like form (Sec. 5.1) */

/* Entry (p, q) of the Cauchy-like matrix with generators G (n x P, row-major)
 * and B (P x m, row-major): sum_l G[p,l] B[l,q] / (x_p - y_q)  (Eq. cauchy-like). */
static cplx cauchy_like_entry(const cplx* x, const cplx* y, const cplx* G, const cplx* B, int64_t m, int64_t P,
                              int64_t p, int64_t q) {
  cplx s = 0.0;
  for (int64_t l = 0; l < P; ++l) s = s + G[p * P + l] * B[l * m + q];
  return s / (x[p] - y[q]);
}

/* RPLU of a Cauchy-like matrix through its generators (Algorithm 3 of Sec. 5.1),
 * with the squared row norms of the residual recomputed exactly from the
 * current generators at every step instead of bounded and rejection-sampled.
 * Each step: d_p = sum_q |S_pq|^2 with S = the residual in generator form;
 * the row is drawn by d, the pivot row r = S(i,:), the column by |r_q|^2 over
 * unpivoted columns, a = r_j, the pivot column c = S(:,j);
 * L(:,t) = c / a (L(i,t) = 1, L(I_prev,t) = 0), U(t,:) = r (U(t,J_prev) = 0);
 * then Eqs. generator_update_g / generator_update_b:
 *   G <- G - (c / a) G(i,:),   B <- B - B(:,j) (r / a),
 * with G(i,:) and B(:,j) set to exact zero.  Draws, redraws, stopping and
 * outputs as oracle_rplu_dense_c128.  G_out / B_out (optional) receive the
 * final generators.  Returns 0, or -1 on an invalid argument. */
int oracle_rplu_cauchy_like(const cplx* x, const cplx* y, const cplx* G0, const cplx* B0, int64_t n, int64_t m,
                            int64_t P, int64_t k, uint64_t seed, int32_t mode, const int64_t* given_I,
                            const int64_t* given_J, double tol, int64_t* piv_I, int64_t* piv_J, cplx* L, cplx* U,
                            double* T_hist, double* row_margin, double* col_margin, cplx* G_out, cplx* B_out,
                            int64_t* k_done) {
  if (n < 0 || m < 0 || P < 1 || k < 0 || k > (n < m ? n : m) || mode == MODE_COMPLETE) return -1;
  cplx* G = (cplx*)malloc(sizeof(cplx) * (size_t)(n * P > 0 ? n * P : 1));
  cplx* B = (cplx*)malloc(sizeof(cplx) * (size_t)(P * m > 0 ? P * m : 1));
  cplx* gi = (cplx*)malloc(sizeof(cplx) * (size_t)P);
  cplx* bj = (cplx*)malloc(sizeof(cplx) * (size_t)P);
  double* d = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* wcol = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  cplx* r = (cplx*)malloc(sizeof(cplx) * (size_t)(m > 0 ? m : 1));
  cplx* c = (cplx*)malloc(sizeof(cplx) * (size_t)(n > 0 ? n : 1));
  char* col_used = (char*)calloc((size_t)(m > 0 ? m : 1), 1);
  char* row_used = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!G || !B || !gi || !bj || !d || !wcol || !r || !c || !col_used || !row_used) {
    free(G); free(B); free(gi); free(bj); free(d); free(wcol); free(r); free(c); free(col_used); free(row_used);
    return -1;
  }
  memcpy(G, G0, sizeof(cplx) * (size_t)(n * P));
  memcpy(B, B0, sizeof(cplx) * (size_t)(P * m));
  memset(L, 0, sizeof(cplx) * (size_t)(n * k));
  memset(U, 0, sizeof(cplx) * (size_t)(k * m));
  double T0 = 0.0;
  int64_t t = 0;
  for (;; ++t) {
    /* exact squared row norms of the current residual */
    for (int64_t p = 0; p < n; ++p) {
      double s = 0.0;
      for (int64_t q = 0; q < m; ++q) s = s + abs2(cauchy_like_entry(x, y, G, B, m, P, p, q));
      d[p] = s;
    }
    double T = sum_in_order(d, n);
    if (t == 0) T0 = T;
    T_hist[t] = T;
    if (t == k) break;
    if (!(T > 0.0) || (tol > 0.0 && T <= tol * tol * T0)) break;
    int64_t i = -1, j = -1;
    double rm = 0.0, cm = 0.0;
    int ok = 0;
    for (int attempt = 0; attempt < MAX_ATTEMPTS && !ok; ++attempt) {
      if (mode == MODE_GIVEN) i = given_I[t];
      else if (mode == MODE_RANDOM) {
        double u1 = oracle_u01(seed, t, 0, attempt);
        i = oracle_inverse_cdf(d, n, u1 * T, T, &rm);
      } else i = argmax_first(d, n);
      for (int64_t q = 0; q < m; ++q) r[q] = cauchy_like_entry(x, y, G, B, m, P, i, q);
      if (mode == MODE_GIVEN) { j = given_J[t]; ok = 1; break; }
      for (int64_t q = 0; q < m; ++q) wcol[q] = col_used[q] ? 0.0 : abs2(r[q]);
      double R = sum_in_order(wcol, m);
      if (!(R > 0.0)) {
        d[i] = 0.0;
        T = sum_in_order(d, n);
        if (!(T > 0.0)) break;
        continue;
      }
      if (mode == MODE_RANDOM) {
        double u2 = oracle_u01(seed, t, 1, attempt);
        j = oracle_inverse_cdf(wcol, m, u2 * R, R, &cm);
      } else j = argmax_first(wcol, m);
      ok = 1;
    }
    if (!ok) break;
    cplx a = r[j];
    for (int64_t p = 0; p < n; ++p) c[p] = cauchy_like_entry(x, y, G, B, m, P, p, j);
    for (int64_t q = 0; q < m; ++q) U[t * m + q] = col_used[q] ? 0.0 : r[q];
    for (int64_t p = 0; p < n; ++p) L[t * n + p] = row_used[p] ? 0.0 : c[p] / a;
    L[t * n + i] = 1.0;
    piv_I[t] = i;
    piv_J[t] = j;
    if (row_margin) row_margin[t] = rm;
    if (col_margin) col_margin[t] = cm;
    row_used[i] = 1;
    col_used[j] = 1;
    /* Eqs. generator_update_g / generator_update_b with the generators of step t */
    for (int64_t l = 0; l < P; ++l) {
      gi[l] = G[i * P + l];
      bj[l] = B[l * m + j];
    }
    for (int64_t p = 0; p < n; ++p) {
      cplx lp = L[t * n + p];
      for (int64_t l = 0; l < P; ++l) G[p * P + l] = G[p * P + l] - lp * gi[l];
    }
    for (int64_t q = 0; q < m; ++q) {
      cplx uq = U[t * m + q] / a;
      for (int64_t l = 0; l < P; ++l) B[l * m + q] = B[l * m + q] - bj[l] * uq;
    }
    for (int64_t l = 0; l < P; ++l) {
      G[i * P + l] = 0.0;
      B[l * m + j] = 0.0;
    }
  }
  *k_done = t;
  if (G_out) memcpy(G_out, G, sizeof(cplx) * (size_t)(n * P));
  if (B_out) memcpy(B_out, B, sizeof(cplx) * (size_t)(P * m));
  free(G); free(B); free(gi); free(bj); free(d); free(wcol); free(r); free(c); free(col_used); free(row_used);
  return 0;
}

/* ------------------------------- row-norm upper bounds (App. C, Sec. 5.1) */

/* Quadtree over 2-D points (complex numbers): a node holds the contiguous
 * range [lo, hi) of the points in tree order and the tight bounding box of
 * those points; it is a leaf when it holds at most `leaf` points or its box
 * has zero extent (coincident points).  Children split the parent's box at
 * its centre into four quadrants, visited in the order (low re, low im),
 * (high re, low im), (low re, high im), (high re, high im); a point on a
 * split line belongs to the high side. */
typedef struct {
  int64_t lo, hi;
  double x0, x1, y0, y1; /* box: re in [x0, x1], im in [y0, y1] */
  int64_t child[4];      /* -1 when absent */
  int leafnode;
} qnode;

typedef struct {
  qnode* nodes;
  int64_t count, cap;
  int64_t* perm; /* tree order -> original index */
} qtree;

static int64_t qt_new(qtree* t) {
  if (t->count == t->cap) {
    t->cap = t->cap ? 2 * t->cap : 64;
    t->nodes = (qnode*)realloc(t->nodes, sizeof(qnode) * (size_t)t->cap);
  }
  return t->count++;
}

static void qt_box(const cplx* pts, const int64_t* perm, int64_t lo, int64_t hi, qnode* nd) {
  nd->x0 = nd->y0 = 1e308;
  nd->x1 = nd->y1 = -1e308;
  for (int64_t q = lo; q < hi; ++q) {
    const double re = creal(pts[perm[q]]), im = cimag(pts[perm[q]]);
    if (re < nd->x0) nd->x0 = re;
    if (re > nd->x1) nd->x1 = re;
    if (im < nd->y0) nd->y0 = im;
    if (im > nd->y1) nd->y1 = im;
  }
}

static int64_t qt_build(qtree* t, const cplx* pts, int64_t lo, int64_t hi, int64_t leaf, int depth) {
  const int64_t id = qt_new(t);
  qnode nd;
  nd.lo = lo;
  nd.hi = hi;
  for (int c = 0; c < 4; ++c) nd.child[c] = -1;
  qt_box(pts, t->perm, lo, hi, &nd);
  nd.leafnode = (hi - lo <= leaf) || (nd.x1 <= nd.x0 && nd.y1 <= nd.y0) || depth >= 60;
  if (!nd.leafnode) {
    const double cx = 0.5 * (nd.x0 + nd.x1), cy = 0.5 * (nd.y0 + nd.y1);
    /* stable partition into the four quadrants */
    int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(hi - lo));
    int64_t start[5];
    int64_t w = 0;
    for (int c = 0; c < 4; ++c) {
      start[c] = lo + w;
      for (int64_t q = lo; q < hi; ++q) {
        const double re = creal(pts[t->perm[q]]), im = cimag(pts[t->perm[q]]);
        const int qc = (re >= cx ? 1 : 0) + (im >= cy ? 2 : 0);
        if (qc == c) tmp[w++] = t->perm[q];
      }
    }
    start[4] = hi;
    memcpy(t->perm + lo, tmp, sizeof(int64_t) * (size_t)(hi - lo));
    free(tmp);
    for (int c = 0; c < 4; ++c)
      if (start[c + 1] > start[c]) nd.child[c] = qt_build(t, pts, start[c], start[c + 1], leaf, depth + 1);
  }
  t->nodes[id] = nd;
  return id;
}

static void qt_make(qtree* t, const cplx* pts, int64_t n, int64_t leaf) {
  t->nodes = NULL;
  t->count = t->cap = 0;
  t->perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t q = 0; q < n; ++q) t->perm[q] = q;
  if (n > 0) qt_build(t, pts, 0, n, leaf, 0);
}

static double box_dmin2(const qnode* a, const qnode* b) {
  double dx = 0.0, dy = 0.0;
  if (a->x1 < b->x0) dx = b->x0 - a->x1;
  else if (b->x1 < a->x0) dx = a->x0 - b->x1;
  if (a->y1 < b->y0) dy = b->y0 - a->y1;
  else if (b->y1 < a->y0) dy = a->y0 - b->y1;
  return dx * dx + dy * dy;
}

static double box_dmax2(const qnode* a, const qnode* b) {
  const double dx1 = fabs(a->x1 - b->x0), dx2 = fabs(b->x1 - a->x0);
  const double dy1 = fabs(a->y1 - b->y0), dy2 = fabs(b->y1 - a->y0);
  const double dx = dx1 > dx2 ? dx1 : dx2, dy = dy1 > dy2 ? dy1 : dy2;
  return dx * dx + dy * dy;
}

/* Collect the target leaves under node t (in tree order). */
static void qt_leaves(const qtree* T, int64_t t, int64_t* out, int64_t* cnt) {
  if (T->nodes[t].leafnode) {
    out[(*cnt)++] = t;
    return;
  }
  for (int c = 0; c < 4; ++c)
    if (T->nodes[t].child[c] >= 0) qt_leaves(T, T->nodes[t].child[c], out, cnt);
}

/* Upper bounds u_i >= ||S(i,:)||^2 for the Cauchy-like matrix of (x, y, G, B)
 * (App. C): target quadtree on x, source quadtree on y, both with at most
 * `leaf` points per leaf; the dual traversal of Algorithm C.1 splits the
 * larger node of a pair until d_max^2 <= nu d_min^2 (then every target leaf
 * under the target node gets the source node with alpha = 1 / d_min^2(source
 * node, leaf)) or both are leaves (then the pair is summed exactly);
 * Algorithm C.2 forms the Gram matrices H_s = sum_{j in s} B(:,j) B(:,j)^*
 * and u_i = sum alpha G(i,:) H_s G(i,:)^* + the exact near-field terms.
 * Columns listed in skip_col (nonzero) are left out of H_s and of the exact
 * terms.  Returns 0, or -1 on an invalid argument. */
int oracle_bh_bounds(const cplx* x, const cplx* y, const cplx* G, const cplx* B, int64_t n, int64_t m, int64_t P,
                     double nu, int64_t leaf, const char* skip_col, double* u) {
  if (n < 1 || m < 1 || P < 1 || !(nu >= 1.0) || leaf < 1) return -1;
  qtree Tt, Ts;
  qt_make(&Tt, x, n, leaf);
  qt_make(&Ts, y, m, leaf);
  /* Gram matrices of every source node (P x P, row-major, Hermitian) */
  cplx* H = (cplx*)calloc((size_t)(Ts.count * P * P), sizeof(cplx));
  for (int64_t s = 0; s < Ts.count; ++s) {
    cplx* h = H + s * P * P;
    for (int64_t q = Ts.nodes[s].lo; q < Ts.nodes[s].hi; ++q) {
      const int64_t j = Ts.perm[q];
      if (skip_col && skip_col[j]) continue;
      for (int64_t a = 0; a < P; ++a)
        for (int64_t b = 0; b < P; ++b) h[a * P + b] = h[a * P + b] + B[a * m + j] * conj(B[b * m + j]);
    }
  }
  for (int64_t i = 0; i < n; ++i) u[i] = 0.0;
  int64_t* leaves = (int64_t*)malloc(sizeof(int64_t) * (size_t)Tt.count);
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * (Tt.count + Ts.count) * 64 + 16));
  int64_t sp = 0;
  stack[sp++] = 0; /* source root */
  stack[sp++] = 0; /* target root */
  while (sp > 0) {
    const int64_t t = stack[--sp], s = stack[--sp];
    const qnode* ns = &Ts.nodes[s];
    const qnode* nt = &Tt.nodes[t];
    const double dmin2 = box_dmin2(ns, nt), dmax2 = box_dmax2(ns, nt);
    if (dmin2 > 0.0 && dmax2 <= nu * dmin2) {
      int64_t cnt = 0;
      qt_leaves(&Tt, t, leaves, &cnt);
      for (int64_t c = 0; c < cnt; ++c) {
        const qnode* nl = &Tt.nodes[leaves[c]];
        const double alpha = 1.0 / box_dmin2(ns, nl);
        const cplx* h = H + s * P * P;
        for (int64_t q = nl->lo; q < nl->hi; ++q) {
          const int64_t i = Tt.perm[q];
          /* G(i,:) H G(i,:)^* */
          cplx acc = 0.0;
          for (int64_t a = 0; a < P; ++a)
            for (int64_t b = 0; b < P; ++b) acc = acc + G[i * P + a] * h[a * P + b] * conj(G[i * P + b]);
          u[i] = u[i] + alpha * creal(acc);
        }
      }
      continue;
    }
    if (ns->leafnode && nt->leafnode) {
      for (int64_t q = nt->lo; q < nt->hi; ++q) {
        const int64_t i = Tt.perm[q];
        for (int64_t r = ns->lo; r < ns->hi; ++r) {
          const int64_t j = Ts.perm[r];
          if (skip_col && skip_col[j]) continue;
          u[i] = u[i] + abs2(cauchy_like_entry(x, y, G, B, m, P, i, j));
        }
      }
      continue;
    }
    const int split_t = !nt->leafnode && (ns->leafnode || (nt->hi - nt->lo) >= (ns->hi - ns->lo));
    if (split_t) {
      for (int c = 0; c < 4; ++c)
        if (nt->child[c] >= 0) { stack[sp++] = s; stack[sp++] = nt->child[c]; }
    } else {
      for (int c = 0; c < 4; ++c)
        if (ns->child[c] >= 0) { stack[sp++] = ns->child[c]; stack[sp++] = t; }
    }
  }
  free(leaves); free(stack); free(H);
  free(Tt.nodes); free(Tt.perm); free(Ts.nodes); free(Ts.perm);
  return 0;
}

/* RPLU of a Cauchy-like matrix through its generators with Algorithm 3's row
 * draw: rejection sampling against the upper bounds of oracle_bh_bounds.
 * Step t, attempt a (a < 64): propose i by the inverse CDF of u with the
 * uniform U01(seed, t, 0, a); form the exact row r = S(i,:) and rho =
 * ||r||^2; accept when V * u_i < rho with V = U01(seed ^ ACC_STREAM, t, 0, a);
 * then draw the column by |r_q|^2 with U01(seed, t, 1, a).  When 64
 * proposals are rejected the step falls back to the exact-norm draw with
 * U01(seed ^ ACC_STREAM, t, 1, 0) (row) and U01(seed ^ ACC_STREAM, t, 1, 1)
 * (column).  Stopping: when t = k, when sum(u) = 0, or when sum(u) <= tol^2
 * T_0 (T_0 the exact initial total; sum(u) >= ||S||_F^2, so the test is
 * conservative; with stop_max the test is max(u) <= tol^2 max(u at step 0),
 * the stopping rule of the CUR-AAA algorithm of Sec. 5.3).  mode 1 is the
 * approximate C2PLU of Sec. 5.1: the row of the largest bound (ties to the
 * smallest index), then the largest entry of its row; a row whose unpivoted
 * entries are all zero gets u_i = 0 and the next largest is tried; the
 * margins are then the relative gaps between the two largest values and
 * acc_margin is 1.  T_hist[t] = sum(u) at step t; T_hist[k_done] is the exact
 * ||S||_F^2 after the last step.  Near-tie measures of step t: row_margin[t]
 * is the smallest row-draw margin over all its proposals (and the fallback
 * draw), acc_margin[t] the smallest |V u_i - rho| / rho over its proposals
 * (how close any acceptance decision came to the other outcome),
 * col_margin[t] that of the column draw.  Factors and generator updates as
 * oracle_rplu_cauchy_like. */
#define ACC_STREAM 0xA0761D6478BD642FULL

static void exact_row_norms(const cplx* x, const cplx* y, const cplx* G, const cplx* B, int64_t n, int64_t m,
                            int64_t P, double* d) {
  for (int64_t p = 0; p < n; ++p) {
    double s = 0.0;
    for (int64_t q = 0; q < m; ++q) s = s + abs2(cauchy_like_entry(x, y, G, B, m, P, p, q));
    d[p] = s;
  }
}

/* Relative gap between the largest and the second largest of w[0..n) (1 when
 * fewer than two are positive): the near-tie measure of an arg-max. */
static double argmax_gap(const double* w, int64_t n, int64_t* arg) {
  double b1 = -1.0, b2 = -1.0;
  int64_t a = -1;
  for (int64_t q = 0; q < n; ++q) {
    if (w[q] > b1) {
      b2 = b1;
      b1 = w[q];
      a = q;
    } else if (w[q] > b2) {
      b2 = w[q];
    }
  }
  *arg = b1 > 0.0 ? a : -1;
  return (b1 > 0.0 && b2 > 0.0) ? (b1 - b2) / b1 : 1.0;
}

int oracle_rplu_cauchy_like_bh(const cplx* x, const cplx* y, const cplx* G0, const cplx* B0, int64_t n, int64_t m,
                               int64_t P, int64_t k, uint64_t seed, double nu, int64_t leaf, double tol, int mode,
                               int stop_max, int64_t* piv_I, int64_t* piv_J, cplx* L, cplx* U, double* T_hist,
                               double* row_margin, double* col_margin, double* acc_margin, int32_t* attempts,
                               int64_t* k_done) {
  if (n < 1 || m < 1 || P < 1 || k < 0 || k > (n < m ? n : m) || !(nu >= 1.0) || leaf < 1) return -1;
  if (mode != 0 && mode != 1) return -1;
  cplx* G = (cplx*)malloc(sizeof(cplx) * (size_t)(n * P));
  cplx* B = (cplx*)malloc(sizeof(cplx) * (size_t)(P * m));
  cplx* gi = (cplx*)malloc(sizeof(cplx) * (size_t)P);
  cplx* bj = (cplx*)malloc(sizeof(cplx) * (size_t)P);
  double* u = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  double* wcol = (double*)malloc(sizeof(double) * (size_t)m);
  cplx* r = (cplx*)malloc(sizeof(cplx) * (size_t)m);
  cplx* c = (cplx*)malloc(sizeof(cplx) * (size_t)n);
  char* col_used = (char*)calloc((size_t)m, 1);
  char* row_used = (char*)calloc((size_t)n, 1);
  memcpy(G, G0, sizeof(cplx) * (size_t)(n * P));
  memcpy(B, B0, sizeof(cplx) * (size_t)(P * m));
  memset(L, 0, sizeof(cplx) * (size_t)(n * k));
  memset(U, 0, sizeof(cplx) * (size_t)(k * m));
  exact_row_norms(x, y, G, B, n, m, P, d);
  const double T0 = sum_in_order(d, n);
  int64_t t = 0;
  double umax0 = 0.0;
  for (;; ++t) {
    if (t == k) break;
    oracle_bh_bounds(x, y, G, B, n, m, P, nu, leaf, NULL, u);
    const double Usum = sum_in_order(u, n);
    double umax = 0.0;
    for (int64_t p = 0; p < n; ++p) umax = u[p] > umax ? u[p] : umax;
    if (t == 0) umax0 = umax;
    T_hist[t] = Usum;
    if (!(Usum > 0.0)) break;
    if (tol > 0.0 && (stop_max ? umax <= tol * tol * umax0 : Usum <= tol * tol * T0)) break;
    int64_t i = -1, j = -1;
    double rm = INFINITY, cm = 0.0, am = INFINITY;
    int ok = 0, att = 0;
    if (mode == 1) {
      /* approximate C2PLU (Sec. 5.1): the row of the largest bound, then the
       * column of the largest entry of that row; a row with no weight left on
       * unpivoted columns is set aside (its bound zeroed) and the next tried */
      for (int a = 0; a < MAX_ATTEMPTS && !ok; ++a) {
        const double g = argmax_gap(u, n, &i);
        if (i < 0) break;
        if (g < rm) rm = g;
        for (int64_t q = 0; q < m; ++q) r[q] = cauchy_like_entry(x, y, G, B, m, P, i, q);
        for (int64_t q = 0; q < m; ++q) wcol[q] = col_used[q] ? 0.0 : abs2(r[q]);
        att = a + 1;
        cm = argmax_gap(wcol, m, &j);
        if (j < 0) {
          u[i] = 0.0;
          continue;
        }
        am = 1.0;
        ok = 1;
      }
      if (!ok) break;
    }
    for (int a = 0; a < MAX_ATTEMPTS && !ok && mode == 0; ++a) {
      double rma = 0.0;
      i = oracle_inverse_cdf(u, n, oracle_u01(seed, t, 0, a) * Usum, Usum, &rma);
      if (i < 0) break;
      if (rma < rm) rm = rma;
      for (int64_t q = 0; q < m; ++q) r[q] = cauchy_like_entry(x, y, G, B, m, P, i, q);
      for (int64_t q = 0; q < m; ++q) wcol[q] = col_used[q] ? 0.0 : abs2(r[q]);
      const double rho = sum_in_order(wcol, m);
      const double V = oracle_u01(seed ^ ACC_STREAM, t, 0, a);
      att = a + 1;
      if (rho > 0.0 && fabs(V * u[i] - rho) / rho < am) am = fabs(V * u[i] - rho) / rho;
      if (!(rho > 0.0) || !(V * u[i] < rho)) continue;
      j = oracle_inverse_cdf(wcol, m, oracle_u01(seed, t, 1, a) * rho, rho, &cm);
      ok = 1;
    }
    if (!ok) {
      /* every proposal rejected (RPLU mode): the exact-norm draw */
      exact_row_norms(x, y, G, B, n, m, P, d);
      const double T = sum_in_order(d, n);
      if (!(T > 0.0)) break;
      double rmf = 0.0;
      i = oracle_inverse_cdf(d, n, oracle_u01(seed ^ ACC_STREAM, t, 1, 0) * T, T, &rmf);
      if (rmf < rm) rm = rmf;
      for (int64_t q = 0; q < m; ++q) r[q] = cauchy_like_entry(x, y, G, B, m, P, i, q);
      for (int64_t q = 0; q < m; ++q) wcol[q] = col_used[q] ? 0.0 : abs2(r[q]);
      const double R = sum_in_order(wcol, m);
      if (!(R > 0.0)) break;
      j = oracle_inverse_cdf(wcol, m, oracle_u01(seed ^ ACC_STREAM, t, 1, 1) * R, R, &cm);
      att = MAX_ATTEMPTS + 1;
    }
    const cplx a_ = r[j];
    for (int64_t p = 0; p < n; ++p) c[p] = cauchy_like_entry(x, y, G, B, m, P, p, j);
    for (int64_t q = 0; q < m; ++q) U[t * m + q] = col_used[q] ? 0.0 : r[q];
    for (int64_t p = 0; p < n; ++p) L[t * n + p] = row_used[p] ? 0.0 : c[p] / a_;
    L[t * n + i] = 1.0;
    piv_I[t] = i;
    piv_J[t] = j;
    if (row_margin) row_margin[t] = rm;
    if (col_margin) col_margin[t] = cm;
    if (acc_margin) acc_margin[t] = am;
    if (attempts) attempts[t] = att;
    row_used[i] = 1;
    col_used[j] = 1;
    for (int64_t l = 0; l < P; ++l) {
      gi[l] = G[i * P + l];
      bj[l] = B[l * m + j];
    }
    for (int64_t p = 0; p < n; ++p) {
      const cplx lp = L[t * n + p];
      for (int64_t l = 0; l < P; ++l) G[p * P + l] = G[p * P + l] - lp * gi[l];
    }
    for (int64_t q = 0; q < m; ++q) {
      const cplx uq = U[t * m + q] / a_;
      for (int64_t l = 0; l < P; ++l) B[l * m + q] = B[l * m + q] - bj[l] * uq;
    }
    for (int64_t l = 0; l < P; ++l) {
      G[i * P + l] = 0.0;
      B[l * m + j] = 0.0;
    }
  }
  *k_done = t;
  exact_row_norms(x, y, G, B, n, m, P, d);
  T_hist[t] = sum_in_order(d, n);
  free(G); free(B); free(gi); free(bj); free(u); free(d); free(wcol); free(r); free(c); free(col_used); free(row_used);
  return 0;
}
