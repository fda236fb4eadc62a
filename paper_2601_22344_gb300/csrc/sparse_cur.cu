// RPLU in CUR form (Algorithm 2, Sec. 4.1) on a sparse matrix (Sec. 4.3: the
// paper's graph and circuit matrices), real FP64.  The matrix is kept as CSR
// (rows) and CSC (columns); nothing dense of size n x m exists.  A residual row
// r = A(i,:) - b^T A(I,:), a residual column c = A(:,j) - A(:,J) e and the
// correction A(:,J) h are gathers: each output walks its own CSC column (or CSR
// row) and subtracts the entries that lie in an earlier pivot row (or column),
// found through row -> pivot and column -> pivot maps.  A row (or column) of
// at most kSpLongDeg entries is walked by a segment of G lanes of a warp (G
// from the mean degree, so that a warp serves several short rows), a longer
// one by a whole CTA; every sum has a fixed order (lane-strided partial sums,
// then a fixed butterfly), runs are bitwise reproducible, and a step reads the
// matrix three times whatever t is.  The matvec g = A u shares its walk of the
// CSR rows with the residual column.
//
// Per step (t = state.cur), with Uc = A(I,J)^{-1} (k x k):
//   k_sp_zero        rhat = 0, ccol = 0
//   k_sp_rmax, k_sp_rpart, k_sp_sample_row   row i by the row norms d (exact
//                    fixed-point draw over the whole grid, grid_draw.cuh)
//   k_sp_rowraw      (1 CTA)  r = A(i,:); b^T = r(J) Uc (double-double)
//   k_sp_rowgather   r_q -= sum over A(:,q)'s entries in pivot rows I_s of b_s A(I_s,q)  (CSC walk)
//   k_sp_cmask, k_sp_cpart, k_sp_sample_col  u = r with pivoted columns masked,
//                    column j by |u|^2 (likewise)
//   k_sp_colraw      (1 CTA)  c = A(:,j); sigma = c_i - b^T c(I); e = Uc c(I)
//   k_sp_colspmv     one CSR walk: g = A u, and l_p = (c_p - sum over A(p,:)'s
//                    entries in pivot columns J_s of e_s A(p,J_s)) / sigma;
//                    l_i = 1, 0 on pivoted rows
//   k_sp_gI, k_sp_h  h = Uc g(I)
//   k_sp_dupdate     w_p = g_p - (the same gather with h); d <- max(0, d - 2 l w + l^2 ||u||^2)
//                    (CSR walk of the rows with l_p != 0: elsewhere d is unchanged exactly)
//   k_sp_core        Uc <- [[Uc + e b^T / sigma, -e / sigma], [-b^T / sigma, 1 / sigma]]
// The core, b, e, sigma and the update are double-double (dd.cuh), so the
// update's rounding stays below the eps cond(A(I,J)) the FP64 entries carry;
// b, e and h enter the gathers as their high parts.
#include "common.cuh"
#include "dd.cuh"
#include "grid_draw.cuh"
#include "kernels.h"
#include "sampler.cuh"

namespace rplu {
namespace {

constexpr int kSVec = 256;
constexpr int kSSmp = 512;  // threads of the draws
constexpr int kSOne = 1024;  // threads of the one-CTA scatter kernels

inline unsigned grid_for(int64_t work, int threads, int num_sms, int per_sm) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// d_p = sum over row p of v^2 (index order); non-finite values end the run
__global__ void __launch_bounds__(kSVec) k_sp_init(SparseCurLaunch a) {
  bool bad = false;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = a.rp[p]; e < a.rp[p + 1]; ++e) s = fma(a.rv[e], a.rv[e], s);
    bad |= !isfinite(s);
    a.d[p] = s;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
    atomicOr(&a.st->err, kErrNonFinite);
    a.st->done = 1;
  }
}

__global__ void __launch_bounds__(kSVec) k_sp_zero(SparseCurLaunch a) {
  if (a.st->done) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.m; q += stride) a.rhat[q] = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += stride) a.ccol[p] = 0.0;
}

// ------------------------------------------------------------- row draw
// the largest row norm's bit pattern (d >= 0: bit order is value order)
__global__ void __launch_bounds__(kGdThreads) k_sp_rmax(SparseCurLaunch a) {
  __shared__ FxScratch sh;
  if (a.st->done) return;
  const double* d = a.d;
  gd_max([d](int64_t p) -> uint64_t { return fx_bits64(d[p]); }, a.n, a.rdraw, sh);
}

// the chunks' exact fixed-point totals of d
__global__ void __launch_bounds__(kGdThreads) k_sp_rpart(SparseCurLaunch a) {
  __shared__ FxScratch sh;
  if (a.st->done) return;
  const double* d = a.d;
  const int Er = fx_scale_f64(*a.rdraw.maxb, a.n);
  gd_part([d, Er](int64_t p) -> u128 { return fx_f64(d[p], Er); }, a.n, a.rdraw, sh);
}

__global__ void __launch_bounds__(kSSmp) k_sp_sample_row(SparseCurLaunch a) {
  __shared__ FxScratch sh;
  JobState* st = a.st;
  if (st->done) return;
  const uint64_t mb = *a.rdraw.maxb;
  __syncthreads();
  if (threadIdx.x == 0) *a.rdraw.maxb = 0;  // zero for the next draw
  const bool redraw = st->redraw != 0;
  const int64_t t = redraw ? st->cur : st->t;
  const int attempt = redraw ? st->attempt + 1 : 0;
  if (!redraw && t >= a.k) {
    __syncthreads();
    if (threadIdx.x == 0) st->skip = 1;
    return;
  }
  if (attempt >= kMaxAttempts) {
    if (threadIdx.x == 0) { st->done = 1; st->k_done = t; }
    return;
  }
  const double* d = a.d;
  const int Er = fx_scale_f64(mb, a.n);
  auto dw = [d, Er](int64_t p) -> u128 { return fx_f64(d[p], Er); };
  u128 Tfx;
  int64_t i;
  if (a.mode == RPLU_PIVOT_RANDOM) {
    i = gd_select(dw, a.n, a.rdraw, true, draw_u53(a.seed, t, 0, attempt), &Tfx, sh);
  } else {
    (void)gd_select(dw, a.n, a.rdraw, false, 0, &Tfx, sh);
    i = a.mode == RPLU_PIVOT_C2 ? fx_block_argmax([d](int64_t p) -> uint64_t { return fx_bits64(d[p]); }, a.n, sh)
                                : a.gI[t];
  }
  const double T_ = fx_to_double(Tfx, Er);
  bool stop = false;
  int32_t err = 0;
  if (attempt == 0) {
    const double T0 = (t == 0) ? T_ : st->T0;
    if (threadIdx.x == 0) {
      a.T_hist[t] = T_;
      if (t == 0) st->T0 = T_;
    }
    stop = !(T_ > 0.0) || (a.tol > 0.0 && T_ <= a.tol * a.tol * T0);
  } else {
    stop = !(T_ > 0.0);
  }
  if (!stop && a.mode == RPLU_PIVOT_GIVEN && (i < 0 || i >= a.n || a.row_used[i])) {
    stop = true;
    err = kErrBadGiven;
  }
  if (!stop && i < 0) stop = true;
  if (threadIdx.x == 0) {
    if (stop) {
      st->done = 1;
      st->k_done = t;
      if (err) atomicOr(&st->err, err);
    } else {
      st->cur = t;
      st->attempt = attempt;
      st->redraw = 0;
      st->skip = 0;
      st->i = i;
    }
  }
}

// r = A(i,:) scattered (into the zeroed r); b_s = sum_p r(J_p) Uc(p, s) in
// double-double
__global__ void __launch_bounds__(kSOne) k_sp_rowraw(SparseCurLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i;
  double* r = a.rhat;
  for (int64_t e = a.rp[i] + threadIdx.x; e < a.rp[i + 1]; e += blockDim.x) r[a.ci[e]] = a.rv[e];
  __syncthreads();
  for (int64_t s = threadIdx.x; s < t; s += blockDim.x) {
    dd acc = dd_from(0.0);
    for (int64_t p = 0; p < t; ++p) {
      const int64_t e = p * a.k + s;
      acc = dd_add(acc, dd_mul_d(dd{a.core[e], a.core_lo[e]}, r[a.J[p]]));
    }
    a.vb[s] = acc.hi;
    a.vb_lo[s] = acc.lo;
  }
}

// Walk of the rows of a compressed index (CSR rows, or CSC columns): for
// every row p that pre(p, leader) admits, the entries e of p are accumulated
// by acc(e, s) into two sums s, and fin(p, s) consumes them.  Rows of at most
// kSpLongDeg entries: a segment of G lanes per row, 32 / G rows per warp at a
// time, lane-strided partial sums, then a butterfly within the segment (the
// whole warp takes part in every shuffle).  Longer rows (the list longs): a
// CTA each, from block nblk_short on, with a fixed block reduction.  pre() is
// evaluated by every lane of the row's segment or CTA and must give them all
// the same answer; only the leader may write in it.
template <int G, typename Pre, typename Acc, typename Fin>
__device__ __forceinline__ void seg_walk(int64_t n, const int64_t* ptr, const int32_t* longs, int64_t n_long,
                                         unsigned nblk_short, const Pre& pre, const Acc& acc, const Fin& fin) {
  __shared__ double2 red[kSVec / 32];
  const int lane = threadIdx.x & 31;
  if (blockIdx.x < nblk_short) {
    constexpr int RPW = 32 / G;  // rows per warp at a time
    const int sl = lane & (G - 1);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)nblk_short * blockDim.x) >> 5;
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {
      const int64_t p = base + lane / G;
      bool walk = false;
      int64_t e0 = 0, e1 = 0;
      if (p < n) {
        e0 = ptr[p];
        e1 = ptr[p + 1];
        if (e1 - e0 <= kSpLongDeg) walk = pre(p, sl == 0);
      }
      double2 sum = make_double2(0.0, 0.0);
      if (walk)
        for (int64_t e = e0 + sl; e < e1; e += G) acc(e, sum);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o);
        sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o);
      }
      if (walk && sl == 0) fin(p, sum);
    }
    return;
  }
  const int64_t nblk_long = (int64_t)gridDim.x - nblk_short;
  for (int64_t idx = (int64_t)blockIdx.x - nblk_short; idx < n_long; idx += nblk_long) {
    const int64_t p = longs[idx];
    const bool walk = pre(p, threadIdx.x == 0);
    if (!walk) continue;
    double2 sum = make_double2(0.0, 0.0);
    for (int64_t e = ptr[p] + threadIdx.x; e < ptr[p + 1]; e += blockDim.x) acc(e, sum);
    for (int o = 16; o > 0; o >>= 1) {
      sum.x += __shfl_xor_sync(0xffffffffu, sum.x, o);
      sum.y += __shfl_xor_sync(0xffffffffu, sum.y, o);
    }
    if (lane == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 tot = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        tot.x += red[w].x;
        tot.y += red[w].y;
      }
      fin(p, tot);
    }
    __syncthreads();
  }
}

// r_q -= sum of b_s A(I_s, q) over column q's entries whose row is the pivot
// row I_s of an earlier step s < t (CSC walk)
template <int G>
__global__ void __launch_bounds__(kSVec) k_sp_rowgather(SparseCurLaunch a, unsigned nblk_short) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur;
  if (t == 0) return;
  const int32_t* ri = a.ri;
  const double* cv = a.cv;
  const int32_t* row_piv = a.row_piv;
  const double* vb = a.vb;
  double* rhat = a.rhat;
  seg_walk<G>(
      a.m, a.cp, a.long_cols, a.n_long_cols, nblk_short, [](int64_t, bool) { return true; },
      [=](int64_t e, double2& s) {
        const int32_t sp = row_piv[ri[e]];
        if (sp >= 0 && sp < t) s.x = fma(vb[sp], cv[e], s.x);
      },
      [=](int64_t q, double2 s) {
        if (s.x != 0.0) rhat[q] -= s.x;
      });
}

// ------------------------------------------------------------- column draw
// u = r with the pivoted columns masked, and the largest |u_q|'s bit pattern
__global__ void __launch_bounds__(kGdThreads) k_sp_cmask(SparseCurLaunch a) {
  __shared__ FxScratch sh;
  if (a.st->done || a.st->skip) return;
  const double* r = a.rhat;
  const uint8_t* col_used = a.col_used;
  double* urow = a.urow;
  gd_max(
      [r, col_used, urow](int64_t q) -> uint64_t {
        const double v = col_used[q] ? 0.0 : r[q];
        urow[q] = v;
        return entry_max_bits(v);
      },
      a.m, a.cdraw, sh);
}

// the chunks' exact fixed-point totals of |u_q|^2
__global__ void __launch_bounds__(kGdThreads) k_sp_cpart(SparseCurLaunch a) {
  __shared__ FxScratch sh;
  if (a.st->done || a.st->skip) return;
  const double* u = a.urow;
  const int Ec = fx_entry_scale<double>(*a.cdraw.maxb, a.m);
  gd_part([u, Ec](int64_t q) -> u128 { return fx_abs2(u[q], Ec); }, a.m, a.cdraw, sh);
}

__global__ void __launch_bounds__(kSSmp) k_sp_sample_col(SparseCurLaunch a) {
  __shared__ FxScratch sh;
  JobState* st = a.st;
  if (st->done || st->skip) return;
  const uint64_t cb = *a.cdraw.maxb;
  __syncthreads();
  if (threadIdx.x == 0) *a.cdraw.maxb = 0;  // zero for the next draw
  const int64_t t = st->cur, i = st->i;
  const int attempt = st->attempt;
  const double* r = a.rhat;
  const uint8_t* col_used = a.col_used;
  const int Ec = fx_entry_scale<double>(cb, a.m);
  const double* u = a.urow;
  auto cw = [u, Ec](int64_t q) -> u128 { return fx_abs2(u[q], Ec); };
  u128 Rfx;
  int64_t j;
  if (a.mode == RPLU_PIVOT_RANDOM) {
    j = gd_select(cw, a.m, a.cdraw, true, draw_u53(a.seed, t, 1, attempt), &Rfx, sh);
  } else {
    (void)gd_select(cw, a.m, a.cdraw, false, 0, &Rfx, sh);
    j = a.mode == RPLU_PIVOT_C2 ? fx_block_argmax(cw, a.m, sh) : a.gJ[t];
  }
  if (a.mode == RPLU_PIVOT_GIVEN) {
    if (j < 0 || j >= a.m || col_used[j]) {
      if (threadIdx.x == 0) { st->done = 1; st->k_done = t; atomicOr(&st->err, kErrBadGiven); }
      return;
    }
  } else if (Rfx == 0 || j < 0) {
    if (threadIdx.x == 0) {
      a.d[i] = 0.0;
      st->redraw = 1;
      st->skip = 1;
    }
    return;
  }
  const double piv = r[j];
  if (piv == 0.0) {
    if (threadIdx.x == 0) { st->done = 1; st->k_done = t; atomicOr(&st->err, kErrZeroPivot); }
    return;
  }
  if (threadIdx.x == 0) {
    a.col_used[j] = 1;
    a.row_used[i] = 1;
    a.row_piv[i] = (int32_t)t;
    a.col_piv[j] = (int32_t)t;
    a.I[t] = i;
    a.J[t] = j;
    st->j = j;
    st->a_re = piv;
    st->a_im = 0.0;
    st->unorm2 = fx_to_double(Rfx, Ec);
    st->t = t + 1;
  }
}

// c = A(:,j) scattered (into the zeroed c); sigma = c_i - sum_q b_q c(I_q)
// (warp 0) and e_p = sum_s Uc(p, s) c(I_s), both in double-double
__global__ void __launch_bounds__(kSOne) k_sp_colraw(SparseCurLaunch a) {
  JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i, j = st->j;
  double* c = a.ccol;
  for (int64_t e = a.cp[j] + threadIdx.x; e < a.cp[j + 1]; e += blockDim.x) c[a.ri[e]] = a.cv[e];
  __syncthreads();
  if (threadIdx.x < 32) {
    dd acc = dd_from(0.0);
    for (int64_t q = threadIdx.x; q < t; q += 32) acc = dd_add(acc, dd_mul_d(dd{a.vb[q], a.vb_lo[q]}, c[a.I[q]]));
    acc = dd_warp_sum(acc);
    const dd sig = dd_add(dd_from(c[i]), dd_neg(acc));
    if (threadIdx.x == 0) {
      if (sig.hi == 0.0) {
        st->done = 1;
        st->k_done = t;
        atomicOr(&st->err, kErrZeroPivot);
      } else {
        st->a_re = sig.hi;
        st->a_im = sig.lo;
      }
    }
  }
  for (int64_t p = threadIdx.x; p < t; p += blockDim.x) {
    dd acc = dd_from(0.0);
    for (int64_t s = 0; s < t; ++s) {
      const int64_t e = p * a.k + s;
      acc = dd_add(acc, dd_mul_d(dd{a.core[e], a.core_lo[e]}, c[a.I[s]]));
    }
    a.ve[p] = acc.hi;
    a.ve_lo[p] = acc.lo;
  }
}

// One walk of the CSR rows: g_p = sum over row p of v u(col) for every row, and
// l_p = (c_p - sum_s e_s A(p, J_s)) / sigma (FP64 division by its high part),
// l_i = 1, 0 on the rows pivoted before
template <int G>
__global__ void __launch_bounds__(kSVec) k_sp_colspmv(SparseCurLaunch a, unsigned nblk_short) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i;
  const double piv = st->a_re;
  const int32_t* ci = a.ci;
  const double* rv = a.rv;
  const double* u = a.urow;
  const int32_t* col_piv = a.col_piv;
  const double* ve = a.ve;
  const uint8_t* row_used = a.row_used;
  const double* ccol = a.ccol;
  double* g = a.g;
  double* lcol = a.lcol;
  seg_walk<G>(
      a.n, a.rp, a.long_rows, a.n_long_rows, nblk_short, [](int64_t, bool) { return true; },
      [=](int64_t e, double2& s) {
        const double v = rv[e];
        const int32_t c = ci[e];
        s.x = fma(v, u[c], s.x);
        const int32_t sp = col_piv[c];
        if (sp >= 0 && sp < t) s.y = fma(ve[sp], v, s.y);
      },
      [=](int64_t p, double2 s) {
        g[p] = s.x;
        // most rows touch neither column j nor a pivot column: a zero numerator
        // gives the signed zero of IEEE division without the (FP64, slow) divide
        const double num = ccol[p] - s.y;
        lcol[p] = row_used[p] ? (p == i ? 1.0 : 0.0) : num == 0.0 ? (piv < 0.0 ? -num : num) : num / piv;
      });
}

// g(I_s), one thread per s
__global__ void __launch_bounds__(kSVec) k_sp_gI(SparseCurLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < t; s += (int64_t)gridDim.x * blockDim.x)
    a.vg[s] = a.g[a.I[s]];
}

// h_p = sum_s Uc(p, s) g(I_s) in double-double (kept as its high part), one warp per p
__global__ void __launch_bounds__(kSVec) k_sp_h(SparseCurLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur;
  const int lane = threadIdx.x & 31;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < t;
       p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    dd acc = dd_from(0.0);
    for (int64_t s = lane; s < t; s += 32) {
      const int64_t e = p * a.k + s;
      acc = dd_add(acc, dd_mul_d(dd{a.core[e], a.core_lo[e]}, a.vg[s]));
    }
    acc = dd_warp_sum(acc);
    if (lane == 0) a.vh[p] = acc.hi;
  }
}

// w_p = g_p - sum_s h_s A(p, J_s); d_p <- max(0, d_p - 2 l_p w_p + l_p^2 ||u||^2),
// d_i = 0.  A row with l_p = 0 keeps d_p exactly (the update adds -2 * 0 * w and
// 0 * ||u||^2), so only the rows with l_p != 0 are walked.
template <int G>
__global__ void __launch_bounds__(kSVec) k_sp_dupdate(SparseCurLaunch a, unsigned nblk_short) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i;
  const double un2 = st->unorm2;
  const int32_t* ci = a.ci;
  const double* rv = a.rv;
  const int32_t* col_piv = a.col_piv;
  const double* vh = a.vh;
  const uint8_t* row_used = a.row_used;
  const double* lcol = a.lcol;
  const double* g = a.g;
  double* d = a.d;
  auto update = [=](int64_t p, double corr) {
    const double w = g[p] - corr;
    const double l = lcol[p];
    const double dn = d[p] - 2.0 * (l * w) + (l * l) * un2;
    d[p] = dn > 0.0 ? dn : 0.0;
  };
  seg_walk<G>(
      a.n, a.rp, a.long_rows, a.n_long_rows, nblk_short,
      [=](int64_t p, bool leader) {
        if (row_used[p]) {
          if (leader && p == i) d[p] = 0.0;
          return false;
        }
        if (lcol[p] == 0.0) return false;
        if (t == 0) {  // no pivot columns yet: nothing to gather
          if (leader) update(p, 0.0);
          return false;
        }
        return true;
      },
      [=](int64_t e, double2& s) {
        const int32_t sp = col_piv[ci[e]];
        if (sp >= 0 && sp < t) s.x = fma(vh[sp], rv[e], s.x);
      },
      [=](int64_t p, double2 s) { update(p, s.x); });
}

// Uc <- [[Uc + e b^T / sigma, -e / sigma], [-b^T / sigma, 1 / sigma]] in
// double-double (in place)
__global__ void __launch_bounds__(kSVec) k_sp_core(SparseCurLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur;
  const dd inv = dd_recip(dd{st->a_re, st->a_im});
  const int64_t t1 = t + 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < t1 * t1; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / t1, s = e - p * t1;
    dd v;
    if (p < t && s < t) {
      const dd ep{a.ve[p], a.ve_lo[p]}, bs{a.vb[s], a.vb_lo[s]};
      v = dd_add(dd{a.core[p * a.k + s], a.core_lo[p * a.k + s]}, dd_mul(dd_mul(ep, bs), inv));
    } else if (p < t) {
      v = dd_neg(dd_mul(dd{a.ve[p], a.ve_lo[p]}, inv));
    } else if (s < t) {
      v = dd_neg(dd_mul(dd{a.vb[s], a.vb_lo[s]}, inv));
    } else {
      v = inv;
    }
    a.core[p * a.k + s] = v.hi;
    a.core_lo[p * a.k + s] = v.lo;
  }
}

__global__ void __launch_bounds__(kSSmp) k_sp_finish(SparseCurLaunch a) {
  __shared__ FxScratch sh;
  JobState* st = a.st;
  const double T = fx_total_f64(a.d, a.n, sh);
  if (threadIdx.x == 0) {
    if (!st->done) {
      st->done = 1;
      st->k_done = st->t;
    }
    a.T_hist[st->k_done] = T;
  }
}

}  // namespace

cudaError_t sparse_cur_init(const SparseCurLaunch& a, cudaStream_t s, HotTimer* tm) {
  k_sp_init<<<grid_for(a.n, kSVec, a.num_sms, 8), kSVec, 0, s>>>(a);
  tm->all_launches += 1;
  return cudaGetLastError();
}

// The short-row blocks of a walk with G lanes per row, and its total grid (one
// more block per long row, at most two per SM).
struct WalkGrid {
  unsigned nshort, total;
};
WalkGrid walk_grid(int64_t rows, int G, int64_t n_long, int num_sms) {
  WalkGrid w;
  w.nshort = grid_for(rows * G, kSVec, num_sms, 8);
  const int64_t nl = n_long < (int64_t)num_sms * 2 ? n_long : (int64_t)num_sms * 2;
  w.total = w.nshort + (unsigned)nl;
  return w;
}

template <int G>
void launch_rowgather(const SparseCurLaunch& a, WalkGrid w, cudaStream_t s) {
  k_sp_rowgather<G><<<w.total, kSVec, 0, s>>>(a, w.nshort);
}
template <int G>
void launch_colspmv(const SparseCurLaunch& a, WalkGrid w, cudaStream_t s) {
  k_sp_colspmv<G><<<w.total, kSVec, 0, s>>>(a, w.nshort);
}
template <int G>
void launch_dupdate(const SparseCurLaunch& a, WalkGrid w, cudaStream_t s) {
  k_sp_dupdate<G><<<w.total, kSVec, 0, s>>>(a, w.nshort);
}
// f<G>(args...) for the segment width G in {2, 4, 8, 16, 32}
#define SP_BY_LANES(G_, f, ...)                  \
  switch (G_) {                                  \
    case 2: f<2>(__VA_ARGS__); break;            \
    case 4: f<4>(__VA_ARGS__); break;            \
    case 8: f<8>(__VA_ARGS__); break;            \
    case 16: f<16>(__VA_ARGS__); break;          \
    default: f<32>(__VA_ARGS__); break;          \
  }

cudaError_t sparse_cur_run(const SparseCurLaunch& a, cudaStream_t s, int64_t steps, HotTimer* tm) {
  const unsigned gz = grid_for(a.n > a.m ? a.n : a.m, kSVec, a.num_sms, 8);
  const WalkGrid wr = walk_grid(a.n, a.row_lanes, a.n_long_rows, a.num_sms);
  const WalkGrid wc = walk_grid(a.m, a.col_lanes, a.n_long_cols, a.num_sms);
  const unsigned gk = grid_for(a.k, kSVec, a.num_sms, 8);
  const unsigned gkw = grid_for(a.k * 32, kSVec, a.num_sms, 8);
  const unsigned gkk = grid_for(a.k * a.k, kSVec, a.num_sms, 8);
  const unsigned grc = (unsigned)a.rdraw.chunks, gcc = (unsigned)a.cdraw.chunks;
  for (int64_t q = 0; q < steps; ++q) {
    k_sp_zero<<<gz, kSVec, 0, s>>>(a);
    k_sp_rmax<<<grc, kGdThreads, 0, s>>>(a);
    k_sp_rpart<<<grc, kGdThreads, 0, s>>>(a);
    k_sp_sample_row<<<1, kSSmp, 0, s>>>(a);
    k_sp_rowraw<<<1, kSOne, 0, s>>>(a);
    SP_BY_LANES(a.col_lanes, launch_rowgather, a, wc, s);
    k_sp_cmask<<<gcc, kGdThreads, 0, s>>>(a);
    k_sp_cpart<<<gcc, kGdThreads, 0, s>>>(a);
    k_sp_sample_col<<<1, kSSmp, 0, s>>>(a);
    k_sp_colraw<<<1, kSOne, 0, s>>>(a);
    tm->begin();
    SP_BY_LANES(a.row_lanes, launch_colspmv, a, wr, s);
    tm->end();
    k_sp_gI<<<gk, kSVec, 0, s>>>(a);
    k_sp_h<<<gkw, kSVec, 0, s>>>(a);
    SP_BY_LANES(a.row_lanes, launch_dupdate, a, wr, s);
    k_sp_core<<<gkk, kSVec, 0, s>>>(a);
    tm->all_launches += 15;
  }
  return cudaGetLastError();
}

cudaError_t sparse_cur_finish(const SparseCurLaunch& a, cudaStream_t s, HotTimer* tm) {
  k_sp_finish<<<1, kSSmp, 0, s>>>(a);
  tm->all_launches += 1;
  return cudaGetLastError();
}

}  // namespace rplu
