// RPLU in CUR form (Algorithm 2, Sec. 4.1) on the multi-level Toeplitz matrix
// of Sec. 4.2: the drifted Gaussian kernel K of Eq. kernel on the Cartesian
// grid {0, h, ..., (N-1) h}^3, A_pq = K(x_p - x_q).  K is a product of three
// one-dimensional Gaussians, so A = T1 (x) T0 (x) T0 exactly, with N x N
// Toeplitz factors given by 2N - 1 taps each; p = (a N + b) N + c.  Entries are
// three tap lookups (taps in shared memory); the matvec A u is three mode
// convolutions, one per axis (3 N^4 FMAs in place of the paper's FFT).  All
// arithmetic is FP64: an FP32 matvec leaves the row-norm estimates of Sec. 4.1
// no better than ~1e-4 of the initial total.
//
// Per step (t = state.cur), with Uc = A(I,J)^{-1} (k x k):
//   k_t3_rmax, k_t3_rpart, k_t3_sample_row   row i by the row norms d (exact
//                    fixed-point draw over the whole grid, grid_draw.cuh)
//   k_t3_b           b^T = A(i,J) Uc
//   k_t3_row         r = A(i,:) - b^T A(I,:)
//   k_t3_cmask, k_t3_cpart, k_t3_sample_col  u = r with pivoted columns masked,
//                    column j by |u|^2 (likewise)
//   k_t3_sigma       (1 warp) sigma = A(i,j) - b^T A(I,j) in double-double
//   k_t3_e           e = Uc A(I,j)
//   k_t3_col         l = (A(:,j) - A(:,J) e) / sigma; l_i = 1, 0 on pivoted rows
//   k_t3_conv x 3    g = A u (u is real, so conj(u) = u)
//   k_t3_gI, k_t3_h  h = Uc g(I)
//   k_t3_dupdate     w = g - A(:,J) h; d <- max(0, d - 2 l w + l^2 ||u||^2)
//   k_t3_core        Uc <- [[Uc + e b^T / sigma, -e / sigma], [-b^T / sigma, 1 / sigma]]
// The core, b, e, sigma and the update are double-double (dd.cuh): the FP64
// update's rounding grows like eps cond(A(I,J))^2, the double-double one stays
// below the eps cond that the FP64 entries carry.  b, e and h enter the
// residual row, column and correction as their high parts.
#include "common.cuh"
#include "dd.cuh"
#include "grid_draw.cuh"
#include "kernels.h"
#include "sampler.cuh"

namespace rplu {
namespace {

constexpr int kTVec = 256;       // threads of the vector kernels
constexpr int kTSmp = 512;       // threads of the draws
constexpr int kTChunk = 256;     // pivots staged in shared memory at a time
constexpr int kTPerThread = 4;   // outputs per thread in the generated kernels
constexpr int kConvTW = 16;      // lines per mode-convolution tile
constexpr int kConvLd = kConvTW + 1;  // padded leading dimension of the tile
constexpr int kConvThreads = 256;
constexpr int kConvRows = 4;     // outputs per thread per pass

struct Dig {
  int a, b, c;
};

__device__ __forceinline__ Dig digits(int64_t p, int N) {
  const int64_t ab = p / N;
  const int64_t a = ab / N;
  return Dig{(int)a, (int)(ab - a * N), (int)(p - ab * N)};
}

// A(p, q) from the digits of p and q; the product in the order (T1 * T0) * T0
__device__ __forceinline__ double entry(const double* t1, const double* t0, int N, Dig p, Dig q) {
  return (t1[p.a - q.a + N - 1] * t0[p.b - q.b + N - 1]) * t0[p.c - q.c + N - 1];
}

__device__ __forceinline__ void load_taps(const Toeplitz3Launch& a, double* s1, double* s0) {
  const int L = 2 * a.N - 1;
  for (int e = threadIdx.x; e < L; e += blockDim.x) {
    s1[e] = a.t1[e];
    s0[e] = a.t0[e];
  }
}

inline unsigned grid_for(int64_t work, int threads, int num_sms, int per_sm) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// ------------------------------------------------------------ initial norms
// r1d[a] = sum_a' T1[a, a']^2, r1d[N + b] = sum_b' T0[b, b']^2 (index order)
__global__ void __launch_bounds__(kTVec) k_t3_rownorm1d(Toeplitz3Launch a) {
  const int N = a.N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * N; e += gridDim.x * blockDim.x) {
    const double* tp = e < N ? a.t1 : a.t0;
    const int r = e < N ? e : e - N;
    double s = 0.0;
    for (int c = 0; c < N; ++c) {
      const double v = tp[r - c + N - 1];
      s += v * v;
    }
    a.r1d[e] = s;
  }
}

// d_p = (r1[a] r0[b]) r0[c]: the row norms of a Kronecker product
__global__ void __launch_bounds__(kTVec) k_t3_init(Toeplitz3Launch a) {
  const int N = a.N;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    const Dig dp = digits(p, N);
    a.d[p] = (a.r1d[dp.a] * a.r1d[N + dp.b]) * a.r1d[N + dp.c];
  }
}

// ------------------------------------------------------------- row draw
// the largest row norm's bit pattern (d >= 0: bit order is value order)
__global__ void __launch_bounds__(kGdThreads) k_t3_rmax(Toeplitz3Launch a) {
  __shared__ FxScratch sh;
  if (a.st->done) return;
  const double* d = a.d;
  gd_max([d](int64_t p) -> uint64_t { return fx_bits64(d[p]); }, a.n, a.rdraw, sh);
}

// the chunks' exact fixed-point totals of d
__global__ void __launch_bounds__(kGdThreads) k_t3_rpart(Toeplitz3Launch a) {
  __shared__ FxScratch sh;
  if (a.st->done) return;
  const double* d = a.d;
  const int Er = fx_scale_f64(*a.rdraw.maxb, a.n);
  gd_part([d, Er](int64_t p) -> u128 { return fx_f64(d[p], Er); }, a.n, a.rdraw, sh);
}

__global__ void __launch_bounds__(kTSmp) k_t3_sample_row(Toeplitz3Launch a) {
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

// b_s = sum_p A(i, J_p) Uc(p, s) in double-double, one thread per s
__global__ void __launch_bounds__(kTVec) k_t3_b(Toeplitz3Launch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int N = a.N;
  const int64_t t = st->cur;
  const Dig di = digits(st->i, N);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < t; s += (int64_t)gridDim.x * blockDim.x) {
    dd acc = dd_from(0.0);
    for (int64_t p = 0; p < t; ++p) {
      const int64_t e = p * a.k + s;
      acc = dd_add(acc, dd_mul_d(dd{a.core[e], a.core_lo[e]}, entry(a.t1, a.t0, N, di, digits(a.J[p], N))));
    }
    a.vb[s] = acc.hi;
    a.vb_lo[s] = acc.lo;
  }
}

// out_q = base(q) - sum_s coef_s A(piv_s, q) (rows of pivots: piv_is_row) or
//         base(q) - sum_s A(q, piv_s) coef_s (columns of pivots), for kTPerThread
// outputs per thread; the pivots' digits and coefficients staged in shared memory.
// `base` returns the generated first term; `fin` consumes each output.
template <bool kPivRows, typename Base, typename Fin>
__device__ __forceinline__ void generated_pass(const Toeplitz3Launch& a, const double* s1, const double* s0,
                                               const int64_t* piv, const double* coef, int64_t t, const Base& base,
                                               const Fin& fin) {
  __shared__ int sa[kTChunk], sb[kTChunk], sc[kTChunk];
  __shared__ double sv[kTChunk];
  const int N = a.N;
  const int64_t span = (int64_t)blockDim.x * kTPerThread;
  for (int64_t q0 = (int64_t)blockIdx.x * span; q0 < a.n; q0 += (int64_t)gridDim.x * span) {
    int64_t q[kTPerThread];
    Dig dq[kTPerThread];
    double acc[kTPerThread];
#pragma unroll
    for (int r = 0; r < kTPerThread; ++r) {
      q[r] = q0 + threadIdx.x + (int64_t)r * blockDim.x;
      dq[r] = digits(q[r] < a.n ? q[r] : 0, N);
      acc[r] = q[r] < a.n ? base(q[r], dq[r]) : 0.0;
    }
    for (int64_t c0 = 0; c0 < t; c0 += kTChunk) {
      const int cnt = (int)min((int64_t)kTChunk, t - c0);
      __syncthreads();
      for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        const Dig dp = digits(piv[c0 + e], N);
        sa[e] = dp.a;
        sb[e] = dp.b;
        sc[e] = dp.c;
        sv[e] = coef[c0 + e];
      }
      __syncthreads();
      for (int e = 0; e < cnt; ++e) {
        const Dig dp{sa[e], sb[e], sc[e]};
        const double v = sv[e];
#pragma unroll
        for (int r = 0; r < kTPerThread; ++r) {
          const double A_ = kPivRows ? entry(s1, s0, N, dp, dq[r]) : entry(s1, s0, N, dq[r], dp);
          acc[r] = fma(-v, A_, acc[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kTPerThread; ++r)
      if (q[r] < a.n) fin(q[r], acc[r]);
  }
}

// r_q = A(i,q) - sum_s b_s A(I_s, q)
__global__ void __launch_bounds__(kTVec) k_t3_row(Toeplitz3Launch a) {
  extern __shared__ double taps[];
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int N = a.N;
  double* s1 = taps;
  double* s0 = taps + (2 * N - 1);
  load_taps(a, s1, s0);
  __syncthreads();
  const int64_t t = st->cur;
  const Dig di = digits(st->i, N);
  double* r = a.rhat;
  generated_pass<true>(
      a, s1, s0, a.I, a.vb, t, [&](int64_t, Dig dq) { return entry(s1, s0, N, di, dq); },
      [&](int64_t q, double v) { r[q] = v; });
}

// ------------------------------------------------------------- column draw
// u = r with the pivoted columns masked, and the largest |u_q|'s bit pattern
__global__ void __launch_bounds__(kGdThreads) k_t3_cmask(Toeplitz3Launch a) {
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
      a.n, a.cdraw, sh);
}

// the chunks' exact fixed-point totals of |u_q|^2
__global__ void __launch_bounds__(kGdThreads) k_t3_cpart(Toeplitz3Launch a) {
  __shared__ FxScratch sh;
  if (a.st->done || a.st->skip) return;
  const double* u = a.urow;
  const int Ec = fx_entry_scale<double>(*a.cdraw.maxb, a.n);
  gd_part([u, Ec](int64_t q) -> u128 { return fx_abs2(u[q], Ec); }, a.n, a.cdraw, sh);
}

__global__ void __launch_bounds__(kTSmp) k_t3_sample_col(Toeplitz3Launch a) {
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
  const int Ec = fx_entry_scale<double>(cb, a.n);
  const double* u = a.urow;
  auto cw = [u, Ec](int64_t q) -> u128 { return fx_abs2(u[q], Ec); };
  u128 Rfx;
  int64_t j;
  if (a.mode == RPLU_PIVOT_RANDOM) {
    j = gd_select(cw, a.n, a.cdraw, true, draw_u53(a.seed, t, 1, attempt), &Rfx, sh);
  } else {
    (void)gd_select(cw, a.n, a.cdraw, false, 0, &Rfx, sh);
    j = a.mode == RPLU_PIVOT_C2 ? fx_block_argmax(cw, a.n, sh) : a.gJ[t];
  }
  if (a.mode == RPLU_PIVOT_GIVEN) {
    if (j < 0 || j >= a.n || col_used[j]) {
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
    a.I[t] = i;
    a.J[t] = j;
    st->j = j;
    st->a_re = piv;
    st->a_im = 0.0;
    st->unorm2 = fx_to_double(Rfx, Ec);
    st->t = t + 1;
  }
}

// sigma = A(i,j) - sum_q b_q A(I_q, j) in double-double (one warp); it replaces
// the FP64 residual entry r_j as the pivot (its high part) and in the core update
__global__ void __launch_bounds__(32) k_t3_sigma(Toeplitz3Launch a) {
  JobState* st = a.st;
  if (st->done || st->skip) return;
  const int N = a.N;
  const int64_t t = st->cur;
  const Dig di = digits(st->i, N), dj = digits(st->j, N);
  dd acc = dd_from(0.0);
  for (int64_t q = threadIdx.x; q < t; q += 32)
    acc = dd_add(acc, dd_mul_d(dd{a.vb[q], a.vb_lo[q]}, entry(a.t1, a.t0, N, digits(a.I[q], N), dj)));
  acc = dd_warp_sum(acc);
  const dd sig = dd_add(dd_from(entry(a.t1, a.t0, N, di, dj)), dd_neg(acc));
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

// e_p = sum_s Uc(p, s) A(I_s, j) in double-double, one warp per p (lanes over s)
__global__ void __launch_bounds__(kTVec) k_t3_e(Toeplitz3Launch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int N = a.N;
  const int64_t t = st->cur;
  const Dig dj = digits(st->j, N);
  const int lane = threadIdx.x & 31;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < t;
       p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    dd acc = dd_from(0.0);
    for (int64_t s = lane; s < t; s += 32) {
      const int64_t e = p * a.k + s;
      acc = dd_add(acc, dd_mul_d(dd{a.core[e], a.core_lo[e]}, entry(a.t1, a.t0, N, digits(a.I[s], N), dj)));
    }
    acc = dd_warp_sum(acc);
    if (lane == 0) {
      a.ve[p] = acc.hi;
      a.ve_lo[p] = acc.lo;
    }
  }
}

// l_p = (A(p,j) - sum_s A(p, J_s) e_s) / sigma (FP64 division by its high part); l_i = 1, 0 on the
// rows pivoted before
__global__ void __launch_bounds__(kTVec) k_t3_col(Toeplitz3Launch a) {
  extern __shared__ double taps[];
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int N = a.N;
  double* s1 = taps;
  double* s0 = taps + (2 * N - 1);
  load_taps(a, s1, s0);
  __syncthreads();
  const int64_t t = st->cur, i = st->i;
  const Dig dj = digits(st->j, N);
  const double piv = st->a_re;
  const uint8_t* used = a.row_used;
  double* lc = a.lcol;
  generated_pass<false>(
      a, s1, s0, a.J, a.ve, t, [&](int64_t, Dig dp) { return entry(s1, s0, N, dp, dj); },
      [&](int64_t p, double v) { lc[p] = used[p] ? (p == i ? 1.0 : 0.0) : v / piv; });
}

// ----------------------------------------------------------- the matvec
// y = T applied along one axis of x viewed as [outer][N][inner]:
//   y[o][jo][w] = sum_j taps[jo - j + N - 1] x[o][j][w].
// A tile holds kConvTW lines of length N: for inner > 1 the lines (o, w0 ..
// w0 + kConvTW) (contiguous in w), for inner == 1 the rows o0 .. o0 + kConvTW
// (each contiguous in j).  Element (j, w) of a tile is x[base + j sj + w sw].
__global__ void __launch_bounds__(kConvThreads) k_t3_conv(const double* __restrict__ x, double* __restrict__ y,
                                                          const double* __restrict__ taps, int N, int64_t outer,
                                                          int64_t inner, const JobState* st) {
  extern __shared__ double sm[];
  if (st->done || st->skip) return;
  const int L = 2 * N - 1;
  double* stap = sm;
  double* tile = sm + (L + 1);
  for (int e = threadIdx.x; e < L; e += blockDim.x) stap[e] = taps[e];
  int64_t base, sj, sw;
  int wcount;
  if (inner == 1) {
    const int64_t o0 = (int64_t)blockIdx.x * kConvTW;
    base = o0 * N;
    sj = 1;
    sw = N;
    wcount = (int)min((int64_t)kConvTW, outer - o0);
  } else {
    const int64_t per_o = (inner + kConvTW - 1) / kConvTW;
    const int64_t o = (int64_t)blockIdx.x / per_o;
    const int64_t w0 = ((int64_t)blockIdx.x - o * per_o) * kConvTW;
    base = o * N * inner + w0;
    sj = inner;
    sw = 1;
    wcount = (int)min((int64_t)kConvTW, inner - w0);
  }
  for (int e = threadIdx.x; e < N * kConvTW; e += blockDim.x) {
    int j, w;
    if (inner == 1) {
      w = e / N;
      j = e - w * N;
    } else {
      j = e / kConvTW;
      w = e - j * kConvTW;
    }
    tile[j * kConvLd + w] = w < wcount ? x[base + (int64_t)j * sj + (int64_t)w * sw] : 0.0;
  }
  __syncthreads();
  const int w = threadIdx.x % kConvTW;
  const int grp = threadIdx.x / kConvTW;
  const int ngrp = blockDim.x / kConvTW;
  for (int jb = grp * kConvRows; jb < N; jb += ngrp * kConvRows) {
    double acc[kConvRows];
    int jo[kConvRows];
#pragma unroll
    for (int r = 0; r < kConvRows; ++r) {
      acc[r] = 0.0;
      jo[r] = min(jb + r, N - 1) + N - 1;  // tap offset; rows past N - 1 are computed and dropped
    }
    for (int j = 0; j < N; ++j) {
      const double xv = tile[j * kConvLd + w];
#pragma unroll
      for (int r = 0; r < kConvRows; ++r) acc[r] = fma(stap[jo[r] - j], xv, acc[r]);
    }
    if (w < wcount) {
#pragma unroll
      for (int r = 0; r < kConvRows; ++r)
        if (jb + r < N) y[base + (int64_t)(jb + r) * sj + (int64_t)w * sw] = acc[r];
    }
  }
}

// g(I_s), one thread per s
__global__ void __launch_bounds__(kTVec) k_t3_gI(Toeplitz3Launch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < t; s += (int64_t)gridDim.x * blockDim.x)
    a.vg[s] = a.g[a.I[s]];
}

// h_p = sum_s Uc(p, s) g(I_s) in double-double (kept as its high part), one warp per p
__global__ void __launch_bounds__(kTVec) k_t3_h(Toeplitz3Launch a) {
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

// w_p = g_p - sum_s A(p, J_s) h_s ; d_p <- max(0, d_p - 2 l_p w_p + l_p^2 ||u||^2)
__global__ void __launch_bounds__(kTVec) k_t3_dupdate(Toeplitz3Launch a) {
  extern __shared__ double taps[];
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int N = a.N;
  double* s1 = taps;
  double* s0 = taps + (2 * N - 1);
  load_taps(a, s1, s0);
  __syncthreads();
  const int64_t t = st->cur, i = st->i;
  const double un2 = st->unorm2;
  const uint8_t* used = a.row_used;
  const double* g = a.g;
  const double* lc = a.lcol;
  double* d = a.d;
  generated_pass<false>(
      a, s1, s0, a.J, a.vh, t, [&](int64_t p, Dig) { return g[p]; },
      [&](int64_t p, double w) {
        if (used[p]) {
          if (p == i) d[p] = 0.0;
          return;
        }
        const double l = lc[p];
        const double dn = d[p] - 2.0 * (l * w) + (l * l) * un2;
        d[p] = dn > 0.0 ? dn : 0.0;
      });
}

// Uc <- [[Uc + e b^T / sigma, -e / sigma], [-b^T / sigma, 1 / sigma]] in
// double-double (in place)
__global__ void __launch_bounds__(kTVec) k_t3_core(Toeplitz3Launch a) {
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

__global__ void __launch_bounds__(kTSmp) k_t3_finish(Toeplitz3Launch a) {
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

__global__ void k_t3_core_out(const double* core, int64_t k, int64_t kd, double* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / k, q = e - p * k;
    out[e] = (p < kd && q < kd) ? core[e] : 0.0;
  }
}

size_t taps_bytes(int N) { return (size_t)2 * (2 * N - 1) * sizeof(double); }
size_t conv_bytes(int N) { return ((size_t)(2 * N) + (size_t)N * kConvLd) * sizeof(double); }

cudaError_t conv(const double* x, double* y, const double* taps, int N, int64_t outer, int64_t inner, const JobState* st,
                 cudaStream_t s) {
  const int64_t blocks = inner == 1 ? (outer + kConvTW - 1) / kConvTW : outer * ((inner + kConvTW - 1) / kConvTW);
  k_t3_conv<<<(unsigned)blocks, kConvThreads, conv_bytes(N), s>>>(x, y, taps, N, outer, inner, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t toeplitz3_init(const Toeplitz3Launch& a, cudaStream_t s, HotTimer* tm) {
  const size_t cb = conv_bytes(a.N);
  if (cb > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_t3_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cb);
    if (e != cudaSuccess) return e;
  }
  k_t3_rownorm1d<<<grid_for(2 * a.N, kTVec, a.num_sms, 1), kTVec, 0, s>>>(a);
  k_t3_init<<<grid_for(a.n, kTVec, a.num_sms, 8), kTVec, 0, s>>>(a);
  tm->all_launches += 2;
  return cudaGetLastError();
}

cudaError_t toeplitz3_cur_run(const Toeplitz3Launch& a, cudaStream_t s, int64_t steps, HotTimer* tm) {
  const int64_t N = a.N, n = a.n;
  const size_t tb = taps_bytes(a.N);
  const unsigned gn = grid_for((n + kTPerThread - 1) / kTPerThread, kTVec, a.num_sms, 8);
  const unsigned gk = grid_for(a.k, kTVec, a.num_sms, 8);
  const unsigned gw = grid_for(a.k * 32, kTVec, a.num_sms, 8);
  const unsigned gkk = grid_for(a.k * a.k, kTVec, a.num_sms, 8);
  const unsigned grc = (unsigned)a.rdraw.chunks, gcc = (unsigned)a.cdraw.chunks;
  for (int64_t q = 0; q < steps; ++q) {
    k_t3_rmax<<<grc, kGdThreads, 0, s>>>(a);
    k_t3_rpart<<<grc, kGdThreads, 0, s>>>(a);
    k_t3_sample_row<<<1, kTSmp, 0, s>>>(a);
    k_t3_b<<<gk, kTVec, 0, s>>>(a);
    k_t3_row<<<gn, kTVec, tb, s>>>(a);
    k_t3_cmask<<<gcc, kGdThreads, 0, s>>>(a);
    k_t3_cpart<<<gcc, kGdThreads, 0, s>>>(a);
    k_t3_sample_col<<<1, kTSmp, 0, s>>>(a);
    k_t3_sigma<<<1, 32, 0, s>>>(a);
    k_t3_e<<<gw, kTVec, 0, s>>>(a);
    k_t3_col<<<gn, kTVec, tb, s>>>(a);
    tm->begin();
    cudaError_t e = conv(a.urow, a.g, a.t1, a.N, 1, N * N, a.st, s);  // along a (T1)
    if (e == cudaSuccess) e = conv(a.g, a.tmp, a.t0, a.N, N, N, a.st, s);  // along b
    if (e == cudaSuccess) e = conv(a.tmp, a.g, a.t0, a.N, N * N, 1, a.st, s);  // along c
    tm->end();
    if (e != cudaSuccess) return e;
    k_t3_gI<<<gk, kTVec, 0, s>>>(a);
    k_t3_h<<<gw, kTVec, 0, s>>>(a);
    k_t3_dupdate<<<gn, kTVec, tb, s>>>(a);
    k_t3_core<<<gkk, kTVec, 0, s>>>(a);
    tm->all_launches += 18;
  }
  return cudaGetLastError();
}

cudaError_t toeplitz3_finish(const Toeplitz3Launch& a, cudaStream_t s, HotTimer* tm) {
  k_t3_finish<<<1, kTSmp, 0, s>>>(a);
  tm->all_launches += 1;
  return cudaGetLastError();
}

cudaError_t toeplitz3_core_out(const double* core, int64_t k, int64_t kd, double* out, int num_sms, cudaStream_t s) {
  k_t3_core_out<<<grid_for(k * k, kTVec, num_sms, 8), kTVec, 0, s>>>(core, k, kd, out);
  return cudaGetLastError();
}

}  // namespace rplu
