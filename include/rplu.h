/*
 * rplu.h -- C-ABI of the GB300 (sm_103a) Randomly Pivoted LU library.
 *
 * Problem (paper: Gilles & Wilber, "Low-Rank Approximation by Randomly Pivoted
 * LU", Sec. 1, Algorithm 1): given A (n x m) and a rank k, return the pivot
 * rows I, pivot columns J and factors L (n x k), U (k x m) of k steps of
 * partial Gaussian elimination
 *     L(:,t) = S(:,j_t) / S(i_t,j_t),  U(t,:) = S(i_t,:),  S <- S - L(:,t) U(t,:)
 * (Eq. residual_update), where the pivot (i_t, j_t) is drawn with probability
 * |S_ij|^2 / ||S||_F^2 (Sec. 1) by the two-stage rule of Sec. 4.1: a row with
 * probability proportional to its squared norm, then a column with probability
 * proportional to the squared entries of that row.  The approximation is
 * A ~ L U; A - L U vanishes on rows I and columns J.
 *
 * Conventions shared by every entry point
 *   - Indices are 0-based.  I[t], J[t] are the pivots in the order drawn.
 *   - Where L and U are returned, L is n x k COLUMN-major (column t at L + t*n)
 *     and U is k x m ROW-major (row t at U + t*m).  Complex data are
 *     interleaved (re, im) pairs.
 *   - Every pointer may be host or device memory (classified with
 *     cudaPointerGetAttributes); host data are staged through the device.  The
 *     caller owns all inputs and outputs; the library owns only its workspace,
 *     allocated stream-ordered (cudaMallocAsync) and freed before return.
 *   - Draws: only `seed` determines them.  The uniform for step t, stage s (0
 *     row, 1 column) and redraw attempt a is the top 53 bits of the SplitMix64
 *     output function (Steele, Lea & Flood 2014) at
 *     seed + 0x9E3779B97F4A7C15 * (1 + 128 t + 2 a + s).  The drawn index is
 *     the smallest one whose prefix sum of the weights exceeds u * total; the
 *     sums are exact (each FP64 weight truncated once to 128-bit fixed point
 *     scaled to the largest weight), so the result does not depend on the
 *     order in which the device adds them.
 *   - Pivoted rows and columns are excluded from later draws; U(t, J_prev) and
 *     L(I_prev, t) are stored as exact zeros and L(i_t, t) = 1.
 *   - Precision: FP32/complex64 data keep the Schur update and the Cauchy
 *     matvecs in FP32 with FP32 accumulation; FP64 is used for the squared row
 *     norms (d), the sampling prefix sums and the pivot division.
 *   - Calls are synchronous with respect to the host: they return after the
 *     work queued on `stream` has finished.  Calls on different streams may
 *     run concurrently.
 *   - Errors are status codes; rplu_last_error() returns a message for the
 *     calling thread.  No C++ exception crosses this boundary.
 */
#ifndef RPLU_H
#define RPLU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RPLU_OK = 0,
  RPLU_ERR_INVALID = 1,    /* bad argument, non-finite input, x_i == y_j, zero forced pivot */
  RPLU_ERR_NOMEM = 2,      /* device workspace could not be allocated */
  RPLU_ERR_CUDA = 3,       /* a CUDA runtime call failed */
  RPLU_ERR_TIMEOUT = 4,    /* a bounded device wait expired (batch scheduler) */
  RPLU_NOT_CONVERGED = 5,  /* rel_tol > 0 was not reached within k steps; outputs valid */
  RPLU_CANCELLED = 6       /* serving: the caller cancelled the request; outputs valid for k_done steps */
} rplu_status;

typedef enum { RPLU_F32 = 0, RPLU_F64 = 1, RPLU_C64 = 2, RPLU_C128 = 3 } rplu_dtype;

typedef enum {
  RPLU_PIVOT_RANDOM = 0,   /* RPLU: the two-stage draw (Sec. 1, Sec. 4.1) */
  RPLU_PIVOT_C2 = 1,       /* complete 2-norm pivoting (Sec. 2): argmax row norm, then argmax in row */
  RPLU_PIVOT_COMPLETE = 2, /* complete pivoting (Sec. 1): argmax |S_ij|; dense form only */
  RPLU_PIVOT_GIVEN = 3     /* pivots supplied in given_I / given_J */
} rplu_pivot;

typedef struct {
  int32_t dtype;           /* rplu_dtype of A (or x, y) and of L, U */
  int32_t pivot;           /* rplu_pivot */
  double rel_tol;          /* > 0: stop once ||S||_F^2 <= rel_tol^2 ||A||_F^2 (dense: exact norm;
                              matrix-free: the running estimate); 0: run exactly k steps */
  void* stream;            /* cudaStream_t; NULL = the legacy default stream */
  const int64_t* given_I;  /* RPLU_PIVOT_GIVEN: k distinct rows (host or device) */
  const int64_t* given_J;  /* RPLU_PIVOT_GIVEN: k distinct columns */
  double* T_hist;          /* optional output, k+1 doubles: ||S^(t)||_F^2 before step t, and after
                              the last step at index k_done (matrix-free: sum of the estimates d) */
  double* d_out;           /* optional output, n doubles: squared row norms after the last step */
  int64_t lda;             /* dense: row stride of A in elements; 0 means m */
  int32_t overwrite_input; /* dense, device A only: use A's storage as the residual S (A is
                              clobbered); ignored when A's rows are not 16-byte aligned */
  int32_t pass_block;      /* dense: steps between write-backs of S, 1..8; 0 = default (6 for
                              F32, 4 for C64, 1 for F64/C128).  Every step reads S once and applies the
                              pending rank-1 updates in registers, in the same order as a
                              write-back every step, so the results do not depend on it. */
  double* prof;            /* optional host array of 4 doubles, accumulated (+=) by the call:
                              [0] device ms spent in the per-step Schur-pass kernel (dense:
                              the fused update; matrix-free: the generated matvec), timed with
                              CUDA events on the call's stream; [1] its launches; [2] all
                              kernel launches of the call; [3] calls */
  double bound_nu;         /* rplu_cauchy_like, RANDOM pivots only.  0: exact squared row norms
                              every step.  >= 1: Algorithm 3's row draw by rejection sampling
                              against the upper bounds of App. C (Barnes-Hut quadtrees with
                              the admissibility factor nu: a source node and a target node
                              interact through the node's Gram matrix when
                              d_max^2 <= nu d_min^2); the paper's experiments use 5 */
  int32_t bound_leaf;      /* most points in a quadtree leaf (App. C, "leaf size L"); 0 = 32 */
  int32_t bound_stop;      /* with bound_nu and rel_tol > 0: 0 = stop when sum(u) <= rel_tol^2 ||A||_F^2;
                              1 = stop when max(u) <= rel_tol^2 max(u at step 0), the stopping rule of
                              the CUR-AAA algorithm (Sec. 5.3) */
  int32_t* attempts;       /* optional output, k int32 (bound_nu >= 1): proposals made at each
                              step; kMaxAttempts + 1 = 65 marks a step drawn by the exact-norm
                              fallback after 64 rejections */
} rplu_opts;

/* Fills *o with defaults: RPLU_F64, RPLU_PIVOT_RANDOM, rel_tol 0, NULL stream. */
void rplu_opts_init(rplu_opts* o);

/*
 * rplu_dense -- dense-form RPLU (Algorithm 1; draw of Sec. 4.1).
 *   A        n x m row-major, row stride o->lda (0 = m), dtype o->dtype.
 *   k        number of steps, 0 <= k <= min(n, m).
 *   I, J     int64[k] outputs (entries past *k_done are set to -1).
 *   L, U     outputs, n x k column-major and k x m row-major (dtype o->dtype);
 *            columns/rows past *k_done are zero.
 *   k_done   host int64: steps performed (< k when the residual reached zero,
 *            rel_tol was met, or 64 redraws found only zero rows).
 * The residual S lives in device memory; each step runs one fused pass over S
 * (rank-1 update, exact zeroing of the pivot row and column, new squared row
 * norms).  A in page-locked host memory with 16-byte aligned rows is read in
 * place by the first kernel over the host link (it must stay unchanged until
 * the call returns); other host memory is copied to the device first.  Errors: RPLU_ERR_INVALID for bad sizes/pointers, non-finite
 * entries of A, a zero forced pivot (GIVEN) or COMPLETE with rel_tol.
 */
rplu_status rplu_dense(const void* A, int64_t n, int64_t m, int64_t k, uint64_t seed, const rplu_opts* o,
                       int64_t* I, int64_t* J, void* L, void* U, int64_t* k_done);

/*
 * rplu_cauchy -- matrix-free RPLU of the Cauchy matrix A_ij = 1/(x_i - y_j)
 * (Sec. 5.1 with displacement rank p = 1, G = B = 1).
 *   x, y     n and m points; real (F32/F64) or complex (C64/C128) per o->dtype.
 *   Outputs  as for rplu_dense.  RPLU_PIVOT_COMPLETE is not supported.
 * A is never stored: the residual row A(i,:) - L(i,:)U and column
 * A(:,j) - L U(:,j) are generated (the LU-form analogue of Algorithm 2,
 * Sec. 4.1), and the squared row norms d are updated by the formula of
 * Sec. 4.1 ("Row norm updates") from one generated matvec A conj(u) per step
 * minus the low-rank correction L (U conj(u)).  The estimate's absolute error
 * is of order eps * ||A_i,:||^2 (eps of the data type), so draws are exact only
 * while ||S||_F^2 / ||A||_F^2 stays well above eps.
 * Errors: RPLU_ERR_INVALID for bad sizes/pointers, non-finite points or x_i == y_j
 * (detected as a non-finite initial row norm).
 */
rplu_status rplu_cauchy(const void* x, const void* y, int64_t n, int64_t m, int64_t k, uint64_t seed,
                        const rplu_opts* o, int64_t* I, int64_t* J, void* L, void* U, int64_t* k_done);

/*
 * rplu_cauchy_cur -- matrix-free RPLU of the Cauchy matrix A_ij = 1/(x_i - y_j)
 * in CUR form (Algorithm 2 as printed, Sec. 4.1): no L or U is kept; the pivot
 * rows A(I,:) and columns A(:,J) are generated again each step, and the core
 * inverse A(I,J)^{-1} is updated by block inversion (Eq.
 * block-inverse-update, O(k^2) per step, FP64), so the device memory is
 * O(k^2 + n + m) instead of O(k(n + m)).  The draws, the row-norm update and
 * the stopping test are those of rplu_cauchy, so for the same seed the pivots
 * are the same up to rounding: A ~ A(:,J) core A(I,:) = L U.
 *   x, y, n, m, k, seed, o   as rplu_cauchy (o->pivot RANDOM, C2 or GIVEN).
 *   I, J     int64[k] outputs (entries past *k_done are -1).
 *   core     output, k x k row-major, FP64 for every data type (double for
 *            real data, complex double for complex data, since an inverse with
 *            the condition number of A(I,J) needs it): core(p, s) multiplies
 *            column J_p on the left and row I_s on the right, i.e. core =
 *            A(I,J)^{-1} for the first *k_done pivots; zero elsewhere.  The
 *            entries it inverts are formed in FP64 from the given points.
 * The block inverse is exact arithmetic's inverse; for rapidly decaying
 * spectra A(I,J) becomes ill-conditioned and the core's rounding error grows
 * with its condition number (Sec. 4.1 notes the same).
 * Errors: as rplu_cauchy.
 */
rplu_status rplu_cauchy_cur(const void* x, const void* y, int64_t n, int64_t m, int64_t k, uint64_t seed,
                            const rplu_opts* o, int64_t* I, int64_t* J, void* core, int64_t* k_done);

/*
 * rplu_toeplitz3_cur -- RPLU in CUR form (Algorithm 2, Sec. 4.1) of the
 * multi-level Toeplitz matrix of Sec. 4.2: the drifted Gaussian kernel of Eq.
 * kernel, K(d) = exp(-((d_1 - delta)^2 + d_2^2 + d_3^2) / (2 sigma^2)), on the
 * grid {0, h, ..., (N-1) h}^3 with h = length / N, A_pq = K(x_p - x_q),
 * n = N^3 rows and columns, row p = (a N + b) N + c for the point (a h, b h, c h)
 * (no quadrature weight).  A is the Kronecker product of three N x N Toeplitz
 * matrices; nothing of size n x n is formed: entries are generated from the
 * factors' taps and the matvec of the row-norm update is three mode
 * convolutions.  Real FP64 throughout.  Device memory O(n + k^2).
 *   N        1..640 grid points per axis (the paper: 128 and 320).
 *   length, delta, sigma  the domain's side, the shift along the first axis and
 *            the standard deviation (the paper: 320, 50, 80); length, sigma > 0.
 *   k        0..N^3 steps; seed: the draws (as rplu_dense).
 *   o        o->pivot RANDOM, C2 or GIVEN (o->given_I/J), o->rel_tol (stop when
 *            the row-norm total <= rel_tol^2 of the initial one), o->stream,
 *            o->T_hist (k + 1 doubles), o->d_out (n doubles: the final row-norm
 *            estimates), o->prof ([0] device ms of the matvecs, each three mode
 *            convolutions, [1] matvecs, [2] all launches, [3] calls); o->dtype
 *            is ignored.
 *   I, J     int64[k] outputs (host or device; entries past *k_done are -1).
 *   core     double[k * k] output, row-major: A(I,J)^{-1} for the first *k_done
 *            pivots (core(p, s) multiplies column J_p on the left and row I_s on
 *            the right), zero elsewhere.  It is kept in double-double through
 *            the block-inverse update (Eq. block-inverse-update), so its error
 *            is of order eps cond(A(I,J)), as with a QR of A(I,J).
 * The row norms are updated by the formula of Sec. 4.1, so their total carries
 * an absolute error of order eps ||A||_F^2.
 * Errors: RPLU_ERR_INVALID for N, k, length, sigma or delta out of range, NULL
 * outputs, another pivot mode, or forced pivots out of range or repeated;
 * RPLU_NOT_CONVERGED (outputs valid) when rel_tol was not reached in k steps.
 */
rplu_status rplu_toeplitz3_cur(int64_t N, double length, double delta, double sigma, int64_t k, uint64_t seed,
                               const rplu_opts* o, int64_t* I, int64_t* J, double* core, int64_t* k_done);

/*
 * rplu_sparse_cur -- RPLU in CUR form (Algorithm 2, Sec. 4.1) of a sparse real
 * matrix (Sec. 4.3: graph and circuit matrices), FP64.  Only the CSR arrays, a
 * CSC copy the library builds, the core and O(n + m) vectors are kept.  The
 * residual rows and columns and the correction of the row-norm update are
 * gathers over the CSC columns / CSR rows in a fixed order, the matvec a CSR
 * SpMV: results are bitwise reproducible.
 *   n, m     1..2^31-2 rows and columns.
 *   row_ptr  int64[n + 1], row_ptr[0] = 0, nondecreasing; nnz = row_ptr[n].
 *   col_idx  int32[nnz]: column indices, strictly increasing within each row
 *            (unique entries; scipy's canonical CSR).
 *   val      double[nnz], finite.  The three arrays in host or device memory;
 *            they are read (and copied) by the call, not kept.
 *   k        0..min(n, m); seed: the draws (as rplu_dense).
 *   o        o->pivot RANDOM, C2 or GIVEN (o->given_I/J), o->rel_tol, o->stream,
 *            o->T_hist, o->d_out (n doubles), o->prof ([0] device ms of the SpMVs,
 *            [1] SpMVs, [2] all launches, [3] calls); o->dtype is ignored.
 *   I, J     int64[k] outputs (entries past *k_done are -1).
 *   core     double[k * k] output, row-major: A(I,J)^{-1} for the first *k_done
 *            pivots (core(p, s) multiplies column J_p on the left and row I_s on
 *            the right), zero elsewhere; kept in double-double as in
 *            rplu_toeplitz3_cur (error of order eps cond(A(I,J))).
 * Errors: RPLU_ERR_INVALID for sizes out of range, NULL pointers, a malformed CSR
 * (row_ptr, an index out of range or not increasing within its row), a
 * non-finite value, another pivot mode or bad forced pivots; RPLU_NOT_CONVERGED
 * (outputs valid) when rel_tol was not reached in k steps.
 */
rplu_status rplu_sparse_cur(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                            int64_t k, uint64_t seed, const rplu_opts* o, int64_t* I, int64_t* J, double* core,
                            int64_t* k_done);

/*
 * rplu_cauchy_like -- RPLU of a Cauchy-like matrix through its generators
 * (Sec. 5.1): A_ij = sum_{l<p} G[i,l] B[l,j] / (x_i - y_j) (Eq. cauchy-like),
 * x_i != y_j, displacement rank 1 <= p <= 4.  Plain Cauchy matrices are
 * G = B = 1 (p = 1); Loewner matrices (f(x_i) - f(y_j)) / (x_i - y_j) have
 * p = 2 (Sec. 5.2).
 *   x, y     n and m points; G n x p row-major, B p x m row-major; all of
 *            dtype o->dtype (real or complex).  G and B are not modified.
 *   Outputs  as for rplu_dense.  RPLU_PIVOT_COMPLETE is not supported.
 * Every residual is Cauchy-like; its generators are updated in O((n+m)p)
 * per step by Eqs. generator_update_g / generator_update_b, so the residual
 * is never stored.  Unlike rplu_cauchy, the squared row norms are recomputed
 * exactly from the generated residual at every step (O(nmp)), so the draws
 * and the stopping test carry no estimate drift.
 * With o->bound_nu >= 1 (Algorithm 3 as printed) the row is drawn instead by
 * rejection sampling against upper bounds u_i >= ||S(i,:)||^2 recomputed each
 * step in O((n + m) p^2 log) from quadtrees built once (App. C, Algorithms
 * C.1 and C.2): step t proposes i ~ u with the uniform (seed, t, 0, a) of
 * attempt a, forms r = S(i,:), and accepts when V u_i < ||r||^2, V the
 * uniform (seed ^ 0xA0761D6478BD642F, t, 0, a); the column is drawn from
 * |r_j|^2 with (seed, t, 1, a).  After 64 rejections the step takes the
 * exact-norm draw with the uniforms (seed ^ 0xA0761D6478BD642F, t, 1, 0 / 1).
 * The law of the pivots is that of the exact-norm form.  T_hist[t] is then
 * sum(u) at step t (the stopping test compares it with rel_tol^2 ||A||_F^2,
 * a conservative test since sum(u) >= ||S||_F^2) and T_hist[k_done] the exact
 * ||S||_F^2 after the last step.
 * With bound_nu and RPLU_PIVOT_C2 the step takes the approximate C2PLU of
 * Sec. 5.1 instead: the row of the largest bound (ties to the smallest
 * index), then the largest entry of that row (a row with no weight left on
 * unpivoted columns is set aside and the next largest bound tried).
 * Errors: as rplu_cauchy; RPLU_ERR_INVALID also for p outside 1..4, for
 * bound_nu in (0, 1) or not finite, for bound_nu with a pivot mode other than
 * RANDOM or C2, and (with bound_nu) for n or m >= 2^31.
 */
rplu_status rplu_cauchy_like(const void* x, const void* y, const void* G, const void* B, int64_t n, int64_t m,
                             int64_t p, int64_t k, uint64_t seed, const rplu_opts* o, int64_t* I, int64_t* J,
                             void* L, void* U, int64_t* k_done);

/*
 * rplu_bh_bounds -- the row-norm upper bounds of App. C for one Cauchy-like
 * matrix (x, y, G, B as rplu_cauchy_like): quadtrees with at most `leaf`
 * points per leaf and interaction lists with admissibility factor nu
 * (Algorithm C.1), then u_i = sum over the aggregated source nodes s of
 * G(i,:) H_s G(i,:)^* / d_min^2(s, leaf of i) plus the exact terms of the
 * near source leaves (Algorithm C.2), H_s = sum_{j in s} B(:,j) B(:,j)^*.
 * Up to rounding ||A(i,:)||^2 <= u_i <= nu ||A(i,:)||^2.
 *   u        output, n doubles (host or device).
 * Uses o->dtype and o->stream only.  Errors: RPLU_ERR_INVALID for bad sizes,
 * NULL pointers, nu < 1 or not finite, leaf < 1, p outside 1..4.
 */
rplu_status rplu_bh_bounds(const void* x, const void* y, const void* G, const void* B, int64_t n, int64_t m,
                           int64_t p, double nu, int64_t leaf, const rplu_opts* o, double* u);

/*
 * rplu_bh_plan_stats -- size of the quadtrees and interaction lists that
 * rplu_bh_bounds and rplu_cauchy_like (bound_nu) build for the points x (n)
 * and y (m) (Algorithm C.1), i.e. the work of one evaluation of the bounds
 * (Algorithm C.2).
 *   stats    output, 6 host int64: [0] target leaves, [1] source nodes,
 *            [2] source leaves, [3] aggregated entries (sum of |A_l|),
 *            [4] exact pairs (sum over target leaves l of |l| times the points
 *            of the source leaves in E_l), [5] most points in a target leaf.
 * Uses o->dtype and o->stream.  Errors as rplu_bh_bounds.
 */
rplu_status rplu_bh_plan_stats(const void* x, const void* y, int64_t n, int64_t m, double nu, int64_t leaf,
                               const rplu_opts* o, int64_t* stats);

/*
 * rplu_cur_aaa -- rational approximation by CUR-AAA (Sec. 5.3, Algorithm
 * "CUR-AAA using RPLU"): r(z) = sum_j w_j f(t_j)/(z - t_j) / sum_j w_j/(z - t_j)
 * (Eq. aaa-barycentric) with support points t_j chosen among the samples by
 * Algorithm 3 on the Loewner matrix of a random split of the samples.
 *   z, f     m >= 2 complex128 samples and values (host or device memory).
 *   eps      > 0: Algorithm 3 stops when max(u) <= eps^2 max(u at step 0).
 *   k_max    >= 1: most support points.
 *   seed     the split (sample i goes to X when pi(i) < ceil(m/2), pi a keyed
 *            Feistel permutation of [0, m) with cycle walking) and the pivot draws.
 *   o        o->pivot RPLU_PIVOT_RANDOM (RPLU) or RPLU_PIVOT_C2 (C2PLU), o->bound_nu
 *            (0 = 5), o->bound_leaf, o->stream; o->dtype must be RPLU_C128.
 *   support  output, k_max int64 (host or device): indices into z of the chosen
 *            support points, the first *k entries written.
 *   w        output, k_max complex128: their barycentric weights (2-norm 1): the
 *            right singular vector of the smallest singular value of the Loewner
 *            matrix (f_i - f(t_j))/(z_i - t_j) over the other samples (Eq. Laaa),
 *            from a Householder QR of that matrix and inverse iteration on R.
 *   k        output (host): number of support points.
 *   which    output (host): 0 when the row pivots (points of X) won, 1 the columns (Y).
 *   err      output (host), 2 doubles: max over the samples of |f - r| for the
 *            row and the column candidates.
 * Returns RPLU_NOT_CONVERGED (outputs valid) when k_max steps did not reach eps.
 * Errors: RPLU_ERR_INVALID for bad sizes, NULL pointers, another dtype or
 * pivot mode, non-finite samples or coincident samples across the split.
 */
rplu_status rplu_cur_aaa(const void* z, const void* f, int64_t m, double eps, int64_t k_max, uint64_t seed,
                         const rplu_opts* o, int64_t* support, void* w, int64_t* k, int32_t* which, double* err);

/*
 * rplu_barycentric -- r(zq) of Eq. aaa-barycentric for k support points t with
 * values ft and weights w (complex128), at nq query points; a query equal to a
 * support point gets that point's value.  All arrays host or device memory;
 * rq: output, nq complex128.  Uses o->stream.  Errors: RPLU_ERR_INVALID for
 * k < 1, nq < 0 or NULL pointers.
 */
rplu_status rplu_barycentric(const void* t, const void* ft, const void* w, int64_t k, const void* zq, int64_t nq,
                             const rplu_opts* o, void* rq);

/* One job of a batch (caller-owned; outputs written in place). */
typedef struct {
  int32_t kind;            /* 0 dense (A), 1 Cauchy (x, y): A_ij = 1/(x_i - y_j) */
  int32_t dtype;           /* RPLU_F32, RPLU_F64 or RPLU_C64 (complex points or entries, interleaved re, im) */
  int64_t n, m, k_max, lda;
  double rel_tol;          /* per-job stopping tolerance (0: exactly k_max steps) */
  uint64_t seed;
  const void* A;           /* kind 0: n x m row-major, row stride lda (0 = m) */
  const void* x;           /* kind 1: n points (real for RPLU_F32/F64, complex for RPLU_C64) */
  const void* y;           /* kind 1: m points */
  int64_t* I;              /* outputs, capacity k_max; entries past k_done are -1 */
  int64_t* J;
  void* L;                 /* n x k_max column-major; only the first k_done columns are written */
  void* U;                 /* k_max x m row-major; only the first k_done rows are written */
  int64_t k_done;          /* output */
  int32_t status;          /* output: rplu_status of this job */
  int32_t memory;          /* where the job's buffers are: 0 = ask CUDA for each pointer, 1 = all in host
                              memory, 2 = all in device memory (a hint that spares the per-pointer
                              queries of large batches; a wrong hint is undefined behaviour), 3 = all in
                              host memory that the device reads and writes in place (as 1 on a device
                              without cudaDevAttrPageableMemoryAccess) */
  double rel_res;          /* output: sqrt(||S||_F^2 / ||A||_F^2) after the last step, from the
                              exactly recomputed squared row norms (NaN for a failed job) */
} rplu_job;

/*
 * rplu_batch -- factor many independent small problems (the off-diagonal
 * Cauchy blocks of a hierarchical matrix, Sec. 5.1, or dense blocks) in one
 * persistent launch per data type.  Each job is the dense-form RPLU of its
 * matrix with its own seed and tolerance.  A Cauchy job runs in the
 * generator form (Sec. 5.1, displacement rank 1): its residual is
 * G_p B_q / (x_p - y_q) with generators updated each step, the exact squared
 * row norms are recomputed from them every step, and nothing of size n m is
 * stored.  Jobs
 * with n or m above 4096 run one after another through the single-job
 * kernels instead.  Results do not depend on the launch shape or on the other
 * jobs of the batch.  A complex64 Cauchy job's entry is conj(z) / |z|^2 with
 * z = x_i - y_j and the correctly rounded reciprocal of |z|^2 (the entry
 * rplu_cauchy generates); its multipliers are FP64 complex quotients.
 *   Pointers may be host or device memory per job (jobs[i].memory may say
 *   which, sparing a query per pointer).  Host jobs are staged through pinned
 *   buffers kept by the library: all their inputs go in one copy and all
 *   their results come back in one, so calls that stage host buffers run one
 *   at a time.  Jobs with memory = 3, on a device that accesses pageable host
 *   memory in place (a coherent host link, e.g. a Grace-attached GPU), skip
 *   the pinned buffers: one kernel gathers their inputs from host memory into
 *   device staging and one writes their results into the host outputs.  The
 *   device's first write to an output page the process has not touched yet
 *   goes through the operating system's fault handling, so this suits output
 *   arrays reused from call to call.  Device staging comes from a library memory pool per device
 *   that keeps up to 8 GiB reserved between calls.
 *   o->pivot may be RANDOM or C2; o->stream selects the stream; o->dtype,
 *   o->rel_tol and the dense-only options are ignored (each job has its own).
 * Returns the worst job status; per-job status in jobs[i].status.  Invalid
 * jobs get RPLU_ERR_INVALID and the others still run.
 */
rplu_status rplu_batch(rplu_job* jobs, int32_t njobs, const rplu_opts* o);

/*
 * Batch plans: the same factorizations prepared once and replayed, for
 * callers that factor the same block structure many times (serving, or new
 * values in the same buffers).  rplu_batch_plan_create checks the jobs, sorts
 * them (largest first), allocates the workspace, picks the launch shape and
 * captures the whole batch -- per data type a counter reset, one persistent
 * launch and the copy of the per-job results to pinned host memory -- into a
 * CUDA graph.
 *   jobs      must stay valid until rplu_batch_plan_destroy; every A, x, y, I, J,
 *             L, U must be device memory, n and m at most 4096.  The inputs may
 *             change between runs (same sizes and addresses); results land in
 *             the job's outputs.
 *   tune      0: fixed launch shape (256 threads, 8-row warp tiles, write-back
 *             every 6 steps, as many CTAs per SM as fit).  1: measured
 *             autotuning -- every candidate shape (128 or 256 threads per
 *             CTA, warp tile rows 4/8, write-back interval 4/6/8, 1..4 CTAs per
 *             SM; the compiled subset for the data type) runs the
 *             whole batch once and the fastest is kept; results are identical
 *             for every shape.
 * rplu_batch_plan_run enqueues one replay on `stream` (asynchronous);
 * rplu_batch_plan_wait waits for the last replay and writes k_done, status
 * and rel_res into the jobs, returning the worst status.
 * rplu_batch_plan_shape reports the shape of the plan's largest group:
 * shape[0] threads per CTA, [1] rows per warp tile, [2] write-back interval,
 * [3] CTAs per SM; *tuned_ms (optional) the measured time of that shape (0
 * without tuning).  Replays of one plan must not overlap.
 */
typedef struct rplu_batch_plan rplu_batch_plan;
rplu_status rplu_batch_plan_create(rplu_job* jobs, int32_t njobs, const rplu_opts* o, int32_t tune,
                                   rplu_batch_plan** plan);
rplu_status rplu_batch_plan_run(rplu_batch_plan* plan, void* stream);
rplu_status rplu_batch_plan_wait(rplu_batch_plan* plan);
rplu_status rplu_batch_plan_shape(const rplu_batch_plan* plan, int32_t shape[4], double* tuned_ms);
void rplu_batch_plan_destroy(rplu_batch_plan* plan);

/*
 * rplu_dense_noalloc -- rplu_dense for callers that cannot let the library
 * allocate device memory (the paper has no counterpart; this is a deployment
 * variant).  Examples: code running while a framework's pooled allocator owns
 * the device, services that reserve all memory at start-up and forbid later
 * allocation, and hosts that must avoid the device-wide synchronisation that
 * allocation and release can imply.
 *   Same arguments and results as rplu_dense, with these differences:
 *   - A, I, J, L, U (and given_I/given_J for RPLU_PIVOT_GIVEN) must be device
 *     memory; nothing is staged.
 *   - All working memory comes from one fixed 32 MiB array inside the library,
 *     present on every GPU that loads it until the process exits.  A problem
 *     whose workspace (about n * m * elem_size plus a few vectors) does not fit
 *     returns RPLU_ERR_NOMEM and writes nothing.
 *   - The array is shared by every call: calls whose GPU work overlaps (e.g.
 *     on two streams at once) race and corrupt each other's results; issue
 *     them on one stream or synchronise in between.  Each call clears what
 *     must start at zero.
 *   - The first call on a device looks up the array's device address; make it
 *     before any stream capture begins.
 *   Failures are reported by status code only (rplu_last_error is not set).
 */
rplu_status rplu_dense_noalloc(const void* A, int64_t n, int64_t m, int64_t k, uint64_t seed, const rplu_opts* o,
                               int64_t* I, int64_t* J, void* L, void* U, int64_t* k_done);

/*
 * Serving sessions -- continuous batching (the paper has no serving layer;
 * this is the deployment of the batched kernel for a stream of requests).
 * Requests of mixed kind, type and size are submitted at any time.  A worker
 * thread admits them in arrival order as device memory (a session arena of
 * hbm_budget bytes) and ring slots allow; one persistent kernel picks admitted
 * requests up in arrival order while it runs, one CTA per request, each
 * factored exactly as by rplu_batch (so results equal the request run alone,
 * for the same seed).  The kernel serves FP32 requests (dense A, or real
 * Cauchy points) and complex64 requests (dense complex A, or complex points;
 * entries as rplu_batch forms them); Cauchy requests run in the generator
 * form, whose per-CTA memory grows with n + m only.  Dense requests with n or
 * m above max_dim or n*m above dense_kernel_cells, and Cauchy requests with n
 * or m above cauchy_max_dim, run on up to large_streams streams of their own,
 * concurrently with the kernel: dense ones through rplu_dense, Cauchy ones
 * through rplu_cauchy_like with unit generators (the residual never stored;
 * exact row norms, or with bound_nu >= 1 Algorithm 3's rejection sampling
 * against Barnes-Hut bounds, the request's rel_res then from one extra
 * exact-norm pass over A).  A finished request frees its input copy and
 * workspace at once; its factors stay in the arena until fetched, so a caller
 * that does not fetch holds memory that later requests may need.
 *   - The caller's input buffers (host or device) must stay valid and
 *     unchanged until the request has left the QUEUED state.
 *   - Latency is measured from submit to the completion seen by the worker.
 */
typedef struct rplu_session rplu_session;

typedef struct {
  int64_t hbm_budget;  /* device bytes for inputs, factors and workspaces; 0 = 80% of free memory */
  int32_t max_jobs;    /* ring slots, i.e. requests admitted to the kernel at once (default 4096) */
  int32_t max_dim;     /* largest n and m of a dense request run by the persistent kernel (default 2048,
                          at most 4096) */
  double idle_us;      /* a kernel CTA that finds no request for this long exits (default 1000); the
                          worker launches CTAs in the place of exited ones when requests wait */
  int32_t pivot;       /* RPLU_PIVOT_RANDOM or RPLU_PIVOT_C2 */
  int32_t large_streams; /* requests above the kernel limits run on this many concurrent streams (default 8) */
  int64_t dense_kernel_cells; /* dense requests with n*m above this also take the large-request
                                 streams (0, the default: max_dim^2, every dense request within
                                 max_dim runs in the persistent kernel) */
  int32_t cauchy_max_dim; /* largest n and m of a Cauchy request run by the persistent kernel
                             (0, the default: 4096; at most 4096) */
  int32_t pad0;
  double bound_nu;     /* Cauchy requests on the large-request streams: 0 (the default) = exact
                          squared row norms every step; >= 1 = Algorithm 3's row draw against the
                          App. C upper bounds with this admissibility factor (rplu_cauchy_like's
                          bound_nu; the paper uses 5), RANDOM pivots, or C2PLU's with bounds */
} rplu_session_opts;

typedef struct {
  int32_t kind;        /* 0 dense (A, row stride lda, 0 = m), 1 Cauchy (x, y) */
  int32_t dtype;       /* RPLU_F32 or RPLU_C64 */
  int64_t n, m, k_max, lda;
  double rel_tol;
  uint64_t seed;
  const void* A;
  const void* x;
  const void* y;
} rplu_request;

enum { RPLU_TICKET_QUEUED = 0, RPLU_TICKET_RUNNING = 1, RPLU_TICKET_DONE = 2, RPLU_TICKET_CANCELLED = 3 };

typedef struct {
  int32_t state;       /* RPLU_TICKET_* */
  int32_t status;      /* rplu_status once DONE or CANCELLED */
  int64_t k_done;
  double rel_res;      /* sqrt(||S||_F^2 / ||A||_F^2) after the last step */
  double latency_ms;   /* submit to completion (NaN before) */
  double queue_ms;     /* submit to admission (NaN before) */
} rplu_ticket_info;

void rplu_session_opts_init(rplu_session_opts* o);
rplu_status rplu_session_create(const rplu_session_opts* o, rplu_session** s);
/* Queue a request; *ticket identifies it.  Errors: RPLU_ERR_INVALID for a malformed request. */
rplu_status rplu_session_submit(rplu_session* s, const rplu_request* r, int64_t* ticket);
rplu_status rplu_session_poll(rplu_session* s, int64_t ticket, rplu_ticket_info* info);
/* Block until the ticket is DONE or CANCELLED (RPLU_ERR_TIMEOUT after timeout_s > 0 seconds). */
rplu_status rplu_session_wait(rplu_session* s, int64_t ticket, double timeout_s, rplu_ticket_info* info);
/* Copy the first k_done pivots and factor columns/rows (L n x k_done column-major, U k_done x m
 * row-major; host or device buffers, NULL to skip one) and release the ticket and its memory. */
rplu_status rplu_session_fetch(rplu_session* s, int64_t ticket, int64_t* I, int64_t* J, void* L, void* U);
/* A queued request is dropped; one running in the kernel stops before its next step; one running on a
 * large-request stream finishes first.  All end in state CANCELLED with status RPLU_CANCELLED. */
rplu_status rplu_session_cancel(rplu_session* s, int64_t ticket);
/* Completion queue: up to max_n tickets that finished (DONE or CANCELLED) since the last call,
 * oldest first, with their info; *count receives how many were written. */
rplu_status rplu_session_completed(rplu_session* s, int64_t* tickets, rplu_ticket_info* infos, int32_t max_n,
                                   int32_t* count);
/* out: [0] completed, [1] queued, [2] running, [3] arena bytes in use, [4] arena bytes,
 *      [5] kernel launches, [6] large requests completed, [7] cancelled */
rplu_status rplu_session_stats(rplu_session* s, double out[8]);
/* Stops the kernel after the requests it is running, then frees everything. */
void rplu_session_destroy(rplu_session* s);

const char* rplu_status_string(rplu_status s);
const char* rplu_last_error(void);  /* thread-local message of the last failure */
int32_t rplu_version(void);         /* major*10000 + minor*100 + patch */

#ifdef __cplusplus
}
#endif

#endif /* RPLU_H */
