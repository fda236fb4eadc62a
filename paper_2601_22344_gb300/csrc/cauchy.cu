// Matrix-free RPLU of the Cauchy matrix A_pq = 1/(x_p - y_q) (paper: Sec. 5.1
// with displacement rank p = 1 and G = B = 1; residual rows/columns as in the
// LU form of Algorithm 2, Sec. 4.1; squared-row-norm update of Sec. 4.1).
// Only x, y, L, U and d are stored; entries of A are generated in registers.
//
// Per step (t = state.cur), three launches:
//   k_cf_pivot_cl    (8-CTA cluster; RPLU_PIVOT_RANDOM)  T = sum d, stop test,
//                             row draw i by d, r = A(i,:) - L(i,0:t) U(0:t,:) on
//                             each CTA's eighth of the columns, column draw j by
//                             |r|^2 masked on J, a = r_j, U(t,:) = u = masked r,
//                             ||u||^2; a row whose masked weights sum to zero is
//                             dropped and redrawn inside the launch
//     (other modes: k_cf_sample_row, k_cf_row, k_cf_sample_col, one CTA for
//      each draw; a zero-weight row sets `redraw` and the next launch sequence
//      repeats step t)
//   k_cf_matvec      (grid)   partial sums of g = A conj(u) over column chunks --
//                             the hot loop; CTA number s also forms
//                             v_s = U(s,:) conj(u), s < t
//   k_cf_coldup      (grid)   per row p (8 lanes for the sums, one thread for the
//                             FP64 finish): c_p = A(p,j) - L(p,0:t) U(0:t,j),
//                             L(p,t) = c_p / a (FP64 division), w_p = g_p - L(p,0:t) v;
//                             d_p <- max(0, d_p - 2 Re(conj(l_p) w_p) + |l_p|^2 ||u||^2),
//                             d_i = 0
#include <algorithm>
#include <type_traits>

#include "cluster.cuh"
#include "common.cuh"
#include "kernels.h"
#include "packed.cuh"
#include "sampler.cuh"

namespace rplu {
namespace {

constexpr int kMvThreads = 256;  // matvec CTA size; also the shared tile width
constexpr int kMvRows = 4;       // rows per matvec thread
constexpr int kSmpThreads = 1024;
constexpr int kVecThreads = 256;

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One generated entry 1/(x - y), rounded reciprocal (residual rows/columns).
__device__ __forceinline__ float gen_entry(float x, float y) { return __frcp_rn(x - y); }
__device__ __forceinline__ double gen_entry(double x, double y) { return 1.0 / (x - y); }
__device__ __forceinline__ cf32 gen_entry(cf32 x, cf32 y) {
  const float zr = x.re - y.re, zi = x.im - y.im;
  const float inv = __frcp_rn(fmaf(zr, zr, zi * zi));
  return cf32{zr * inv, -zi * inv};
}
__device__ __forceinline__ cf64 gen_entry(cf64 x, cf64 y) {
  const double zr = x.re - y.re, zi = x.im - y.im;
  const double inv = 1.0 / fma(zr, zr, zi * zi);
  return cf64{zr * inv, -zi * inv};
}

// a * conj(b) accumulated: acc += a conj(b)
__device__ __forceinline__ void mac_conj(float a, float b, float& ar, float&) { ar = fmaf(a, b, ar); }
__device__ __forceinline__ void mac_conj(double a, double b, double& ar, double&) { ar = fma(a, b, ar); }
__device__ __forceinline__ void mac_conj(cf32 a, cf32 b, float& ar, float& ai) {
  ar = fmaf(a.im, b.im, fmaf(a.re, b.re, ar));
  ai = fmaf(-a.re, b.im, fmaf(a.im, b.re, ai));
}
__device__ __forceinline__ void mac_conj(cf64 a, cf64 b, double& ar, double& ai) {
  ar = fma(a.im, b.im, fma(a.re, b.re, ar));
  ai = fma(-a.re, b.im, fma(a.im, b.re, ai));
}

template <typename T> struct TileElem;  // (y_q, u_q) staged in shared memory
template <> struct TileElem<float> { float y, u; };
template <> struct TileElem<double> { double y, u; };
template <> struct alignas(16) TileElem<cf32> { float yr, yi, ur, ui; };
template <> struct alignas(16) TileElem<cf64> { double yr, yi, ur, ui; };

__device__ __forceinline__ TileElem<float> make_tile(float y, float u) { return {y, u}; }
__device__ __forceinline__ TileElem<double> make_tile(double y, double u) { return {y, u}; }
__device__ __forceinline__ TileElem<cf32> make_tile(cf32 y, cf32 u) { return {y.re, y.im, u.re, u.im}; }
__device__ __forceinline__ TileElem<cf64> make_tile(cf64 y, cf64 u) { return {y.re, y.im, u.re, u.im}; }

// The matvec's chunk partials: the chunk sums, accumulated in the working
// precision, stored as they are (FP32 pairs for FP32 types, FP64 pairs else).
template <typename T>
using PartT = typename std::conditional<sizeof(typename Traits<T>::real) == 4, float2, double2>::type;

__device__ __forceinline__ void split(float v, float& r, float& i) { r = v; i = 0.f; }
__device__ __forceinline__ void split(double v, double& r, double& i) { r = v; i = 0.0; }
__device__ __forceinline__ void split(cf32 v, float& r, float& i) { r = v.re; i = v.im; }
__device__ __forceinline__ void split(cf64 v, double& r, double& i) { r = v.re; i = v.im; }

// v_s = U(s,:) conj(u) for s < t, formed by the matvec's CTAs: CTA number L
// (linear index over the grid) takes s = L, L + (grid size), ...; each thread
// sums its columns q = tid, tid + blockDim.x, ... in the working precision,
// then the CTA combines the threads' partials in FP64 by a fixed tree.  No CTA
// waits for another; a CTA with an s reads one row of U and u (about m * 2w
// bytes) besides its matvec tile.
template <typename T>
__device__ void cf_vproj_rows(const CauchyLaunch& a) {
  using real = typename Traits<T>::real;
  __shared__ double red[2][kMvThreads / 32];
  const int64_t t = a.st->cur;
  const T* U = (const T*)a.U;
  const T* u = (const T*)a.urow;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t nblk = (int64_t)gridDim.x * gridDim.y;
  for (int64_t s = (int64_t)blockIdx.y * gridDim.x + blockIdx.x; s < t; s += nblk) {
    real vr = 0, vi = 0;
    for (int64_t q = threadIdx.x; q < a.m; q += blockDim.x) mac_conj(U[s * a.m + q], u[q], vr, vi);
    double dr = (double)vr, di = (double)vi;
    for (int o = 16; o > 0; o >>= 1) {
      dr += __shfl_xor_sync(0xffffffffu, dr, o);
      di += __shfl_xor_sync(0xffffffffu, di, o);
    }
    __syncthreads();
    if (lane == 0) {
      red[0][wid] = dr;
      red[1][wid] = di;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0.0, si = 0.0;
      for (int w = 0; w < kMvThreads / 32; ++w) {
        sr += red[0][w];
        si += red[1][w];
      }
      ((T*)a.vproj)[s] = from_d<T>(sr, si);  // in the working precision, as k_cf_coldup uses it
    }
  }
}

// ------------------------------------------------------------- matvec
// part[c*n + p] = sum over column chunk c of A_pq conj(u_q)        (kNorm false)
//               = sum over column chunk c of |A_pq|^2 in .re       (kNorm true)
// Each thread owns kMvRows rows; (y_q, u_q) tiles are broadcast from shared
// memory; accumulation in the working precision, chunk results in FP64.
template <typename T, bool kNorm>
__global__ void __launch_bounds__(kMvThreads) k_cf_matvec(CauchyLaunch a) {
  using real = typename Traits<T>::real;
  constexpr bool C = Traits<T>::kComplex;
  if (!kNorm && (a.st->done || a.st->skip)) return;
  if constexpr (std::is_same<T, cf32>::value) {
    // complex64: the same arithmetic two rows at a time in packed f32x2
    // instructions; the column's values are staged duplicated ({v, v}):
    // y_re, y_im, u_re, u_im, -u_re, -u_im
    constexpr int NP = kMvRows / 2;
    __shared__ float2 tv[6][kMvThreads];
    const cf32* x = (const cf32*)a.x;
    const cf32* y = (const cf32*)a.y;
    const cf32* u = (const cf32*)a.urow;
    const int64_t row0 = (int64_t)blockIdx.x * (kMvThreads * kMvRows) + threadIdx.x;
    float2 xr2[NP], xi2[NP], gr2[NP], gi2[NP];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      const int64_t p0 = row0 + (int64_t)(2 * h) * kMvThreads, p1 = p0 + kMvThreads;
      const cf32 x0 = p0 < a.n ? x[p0] : x[0], x1 = p1 < a.n ? x[p1] : x[0];
      xr2[h] = make_float2(x0.re, x1.re);
      xi2[h] = make_float2(x0.im, x1.im);
      gr2[h] = make_float2(0.f, 0.f);
      gi2[h] = make_float2(0.f, 0.f);
    }
    const int64_t chunk = (a.m + a.nchunk - 1) / a.nchunk;
    const int64_t q0 = (int64_t)blockIdx.y * chunk;
    const int64_t q1 = min(a.m, q0 + chunk);
    for (int64_t qt = q0; qt < q1; qt += kMvThreads) {
      const int cnt = (int)min((int64_t)kMvThreads, q1 - qt);
      __syncthreads();
      if ((int)threadIdx.x < cnt) {
        const int64_t q = qt + threadIdx.x;
        const cf32 yq = y[q];
        const cf32 uq = kNorm ? cf32{0.f, 0.f} : u[q];
        tv[0][threadIdx.x] = f2_splat(yq.re);
        tv[1][threadIdx.x] = f2_splat(yq.im);
        tv[2][threadIdx.x] = f2_splat(uq.re);
        tv[3][threadIdx.x] = f2_splat(uq.im);
        tv[4][threadIdx.x] = f2_splat(-uq.re);
        tv[5][threadIdx.x] = f2_splat(-uq.im);
      }
      __syncthreads();
      for (int qq = 0; qq < cnt; ++qq) {
        const float2 yr = tv[0][qq], yi = tv[1][qq];
#pragma unroll
        for (int h = 0; h < NP; ++h) {
          const float2 zr = f2_sub(xr2[h], yr), zi = f2_sub(xi2[h], yi);
          const float2 s2 = f2_fma(zr, zr, f2_mul(zi, zi));
          const float2 inv = make_float2(rcp_approx(s2.x), rcp_approx(s2.y));
          if constexpr (kNorm) {
            gr2[h] = f2_fma(inv, make_float2(1.f, 1.f), gr2[h]);
          } else {
            // A conj(u) = (zr - i zi)(ur - i ui) / |z|^2
            const float2 tr = f2_fma(zr, tv[2][qq], f2_mul(zi, tv[5][qq]));   // zr ur - zi ui
            const float2 nti = f2_fma(zr, tv[5][qq], f2_mul(zi, tv[4][qq]));  // -(zr ui + zi ur)
            gr2[h] = f2_fma(tr, inv, gr2[h]);
            gi2[h] = f2_fma(nti, inv, gi2[h]);
          }
        }
      }
    }
    float2* part = (float2*)a.part + (int64_t)blockIdx.y * a.n;
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      const int64_t p0 = row0 + (int64_t)(2 * h) * kMvThreads, p1 = p0 + kMvThreads;
      if (p0 < a.n) part[p0] = make_float2(gr2[h].x, gi2[h].x);
      if (p1 < a.n) part[p1] = make_float2(gr2[h].y, gi2[h].y);
    }
    if constexpr (!kNorm) {
      if (a.U) cf_vproj_rows<T>(a);
    }
    return;
  }
  __shared__ TileElem<T> tile[kMvThreads];
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  const T* u = (const T*)a.urow;
  const int64_t row0 = (int64_t)blockIdx.x * (kMvThreads * kMvRows) + threadIdx.x;
  real xr[kMvRows], xi[kMvRows], gr[kMvRows], gi[kMvRows];
#pragma unroll
  for (int r = 0; r < kMvRows; ++r) {
    const int64_t p = row0 + (int64_t)r * kMvThreads;
    const T xv = p < a.n ? x[p] : x[0];
    split(xv, xr[r], xi[r]);
    gr[r] = 0;
    gi[r] = 0;
  }
  const int64_t chunk = (a.m + a.nchunk - 1) / a.nchunk;
  const int64_t q0 = (int64_t)blockIdx.y * chunk;
  const int64_t q1 = min(a.m, q0 + chunk);
  for (int64_t qt = q0; qt < q1; qt += kMvThreads) {
    const int cnt = (int)min((int64_t)kMvThreads, q1 - qt);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      const int64_t q = qt + threadIdx.x;
      tile[threadIdx.x] = make_tile(y[q], kNorm ? zero_v<T>() : u[q]);
    }
    __syncthreads();
    for (int qq = 0; qq < cnt; ++qq) {
      const TileElem<T> e = tile[qq];
#pragma unroll
      for (int r = 0; r < kMvRows; ++r) {
        if constexpr (C) {
          const real zr = xr[r] - e.yr, zi = xi[r] - e.yi;
          const real s = zr * zr + zi * zi;
          real inv;
          if constexpr (sizeof(real) == 4) inv = rcp_approx(s);
          else inv = 1.0 / s;
          if constexpr (kNorm) {
            gr[r] += inv;
          } else {
            // A conj(u) = (zr - i zi)(ur - i ui) / |z|^2
            const real tr = zr * e.ur - zi * e.ui;
            const real ti = zr * e.ui + zi * e.ur;
            gr[r] = tr * inv + gr[r];
            gi[r] = gi[r] - ti * inv;
          }
        } else {
          const real z = xr[r] - e.y;
          real inv;
          if constexpr (sizeof(real) == 4) inv = rcp_approx(z);
          else inv = 1.0 / z;
          if constexpr (kNorm) gr[r] = inv * inv + gr[r];
          else gr[r] = e.u * inv + gr[r];
        }
      }
    }
  }
  PartT<T>* part = (PartT<T>*)a.part + (int64_t)blockIdx.y * a.n;
#pragma unroll
  for (int r = 0; r < kMvRows; ++r) {
    const int64_t p = row0 + (int64_t)r * kMvThreads;
    if (p < a.n) part[p] = PartT<T>{gr[r], gi[r]};
  }
  if constexpr (!kNorm) {
    if (a.U) cf_vproj_rows<T>(a);
  }
}

// d_p = sum_c part[c][p] (initial squared row norms, FP64 sum); non-finite -> invalid input
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cf_norm_reduce(CauchyLaunch a) {
  const PartT<T>* part = (const PartT<T>*)a.part;
  bool bad = false;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < a.nchunk; ++c) s += (double)part[(int64_t)c * a.n + p].x;
    bad |= !isfinite(s);
    a.d[p] = s;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) {
    atomicOr(&a.st->err, kErrNonFinite);
    a.st->done = 1;
  }
}

// ------------------------------------------------------------- row draw
__global__ void __launch_bounds__(kSmpThreads) k_cf_sample_row(CauchyLaunch a) {
  __shared__ FxScratch sh;
  JobState* st = a.st;
  if (st->done) return;
  const bool redraw = st->redraw != 0;
  const int64_t t = redraw ? st->cur : st->t;
  const int attempt = redraw ? st->attempt + 1 : 0;
  if (!redraw && t >= a.k) {  // all steps done: this launch sequence is idle
    __syncthreads();
    if (threadIdx.x == 0) st->skip = 1;
    return;
  }
  if (attempt >= kMaxAttempts) {
    if (threadIdx.x == 0) { st->done = 1; st->k_done = t; }
    return;
  }
  const double* d = a.d;
  uint64_t mb = max_bits_f64(d, a.n);
  mb = block_max_u64(mb, sh);
  const int Er = fx_scale_f64(mb, a.n);
  auto dw = [d, Er](int64_t p) -> u128 { return fx_f64(d[p], Er); };
  u128 Tfx;
  int64_t i;
  if (a.mode == RPLU_PIVOT_RANDOM) {
    i = fx_block_draw(dw, a.n, draw_u53(a.seed, t, 0, attempt), true, &Tfx, sh);
  } else {
    (void)fx_block_draw(dw, a.n, 0, false, &Tfx, sh);
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

// r = A(i,:) - L(i,0:t) U(0:t,:)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cf_row(CauchyLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  const T* L = (const T*)a.L;
  const T* U = (const T*)a.U;
  T* r = (T*)a.rhat;
  const T xi = x[i];
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.m; q += (int64_t)gridDim.x * blockDim.x) {
    T acc = gen_entry(xi, y[q]);
    for (int64_t s = 0; s < t; ++s) acc = fms(acc, L[s * a.n + i], U[s * a.m + q]);
    r[q] = acc;
  }
}

// ------------------------------------------------------------- column draw
// u = r with pivoted columns masked, written to U(t,:) and the staging row;
// j drawn by |u_q|^2 (exact fixed point); ||u||^2 is the exact total, rounded.
template <typename T>
__global__ void __launch_bounds__(kSmpThreads) k_cf_sample_col(CauchyLaunch a) {
  __shared__ FxScratch sh;
  JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i;
  const int attempt = st->attempt;
  const T* r = (const T*)a.rhat;
  const uint8_t* col_used = a.col_used;
  T* urow = (T*)a.urow;
  T* U = a.U ? (T*)a.U + t * a.m : nullptr;  // the CUR form keeps no U
  uint64_t cb = 0;
  for (int64_t q = threadIdx.x; q < a.m; q += blockDim.x) {
    const T v = col_used[q] ? zero_v<T>() : r[q];
    urow[q] = v;
    if (U) U[q] = v;
    const uint64_t b = entry_max_bits(v);
    cb = b > cb ? b : cb;
  }
  cb = block_max_u64(cb, sh);  // also orders the urow writes before the reads below
  const int Ec = fx_entry_scale<T>(cb, a.m);
  const T* u = urow;
  auto cw = [u, Ec](int64_t q) -> u128 { return fx_abs2(u[q], Ec); };
  u128 Rfx;
  int64_t j;
  if (a.mode == RPLU_PIVOT_RANDOM) {
    j = fx_block_draw(cw, a.m, draw_u53(a.seed, t, 1, attempt), true, &Rfx, sh);
  } else {
    (void)fx_block_draw(cw, a.m, 0, false, &Rfx, sh);
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
  double ar, ai;
  to_d(r[j], ar, ai);
  if (ar == 0.0 && ai == 0.0) {
    if (threadIdx.x == 0) { st->done = 1; st->k_done = t; atomicOr(&st->err, kErrZeroPivot); }
    return;
  }
  if (threadIdx.x == 0) {
    a.col_used[j] = 1;
    a.row_used[i] = 1;
    a.I[t] = i;
    a.J[t] = j;
    st->j = j;
    st->a_re = ar;
    st->a_im = ai;
    st->unorm2 = fx_to_double(Rfx, Ec);
    st->t = t + 1;
  }
}

// ------------------------------------------------------ RANDOM-mode pivot
// The whole pivot choice of one step on a cluster of kCl CTAs (cluster.cuh):
// CTA c owns rows [c RS, (c+1) RS) of d and columns [c CS, (c+1) CS) of the
// residual row.  Row draw by d, residual row on each CTA's columns, column draw
// by |u|^2; partial maxima and exact fixed-point sums are exchanged through
// distributed shared memory, so the draws equal the one-CTA draws of
// k_cf_sample_row / k_cf_sample_col bit for bit.
constexpr int kCfLi = 256;  // L(i, s) values staged in shared memory at a time

template <typename T>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClThreads) k_cf_pivot_cl(CauchyLaunch a) {
  __shared__ FxScratch sh;
  __shared__ ClShared x;
  __shared__ T Li[kCfLi];
  JobState* st = a.st;
  if (st->done) return;  // same value in every CTA: nothing writes it before the final barrier
  const uint32_t rank = cl_rank();
  const int64_t t = st->t;
  if (t >= a.k) {  // every step done: this launch sequence is idle
    if (rank == 0 && threadIdx.x == 0) st->skip = 1;
    return;
  }
  const T* xv = (const T*)a.x;
  const T* yv = (const T*)a.y;
  const T* L = (const T*)a.L;
  T* U = (T*)a.U;
  double* d = a.d;
  const uint8_t* col_used = a.col_used;
  const int64_t RS = (a.n + kCl - 1) / kCl;
  const int64_t rlo = min(a.n, (int64_t)rank * RS), rlen = min(a.n, rlo + RS) - rlo;
  const int64_t CS = (a.m + kCl - 1) / kCl;
  const int64_t qlo = min(a.m, (int64_t)rank * CS), qhi = min(a.m, qlo + CS);

  int ex = 0;  // exchanges so far (selects the buffer)
  const uint64_t gmb = cl_max(max_bits_f64(d + rlo, rlen), x, sh, rank, ex);
  const int Er = fx_scale_f64(gmb, a.n);
  // d is read through L2: a redraw zeroes an entry between two passes over it
  auto dw = [d, Er](int64_t p) -> u128 { return fx_f64(__ldcg(d + p), Er); };
  T* r = (T*)a.rhat;
  T* u = (T*)a.urow;
  T* Ut = U + t * a.m;
  int64_t i = -1, j = -1;
  bool ok = false;
  u128 Rfx = 0;
  int Ec = 0;
  for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
    u128 Tfx;
    i = cl_draw(dw, rlo, rlen, draw_u53(a.seed, t, 0, attempt), &Tfx, x, sh, rank, ex);
    const double T_ = fx_to_double(Tfx, Er);
    if (attempt == 0) {
      const double T0 = (t == 0) ? T_ : st->T0;
      if (rank == 0 && threadIdx.x == 0) {
        a.T_hist[t] = T_;
        if (t == 0) st->T0 = T_;
      }
      if (!(T_ > 0.0) || (a.tol > 0.0 && T_ <= a.tol * a.tol * T0)) break;
    } else if (!(T_ > 0.0)) {
      break;
    }
    if (i < 0) break;
    // r = A(i,:) - L(i,0:t) U(0:t,:) on this CTA's columns, in the order of k_cf_row
    const T xi = xv[i];
    uint64_t cb = 0;
    for (int64_t q0 = qlo; q0 < qhi; q0 += kClThreads) {
      const int64_t q = q0 + threadIdx.x;
      const bool in = q < qhi;
      T acc = in ? gen_entry(xi, yv[q]) : zero_v<T>();
      for (int64_t s0 = 0; s0 < t; s0 += kCfLi) {
        const int cnt = (int)min((int64_t)kCfLi, t - s0);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt; e += kClThreads) Li[e] = L[(s0 + e) * a.n + i];
        __syncthreads();
        if (in) {
          // eight independent loads in flight ahead of the (ordered) FMA chain
          int e = 0;
          for (; e + 8 <= cnt; e += 8) {
            T uv[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) uv[h] = U[(s0 + e + h) * a.m + q];
#pragma unroll
            for (int h = 0; h < 8; ++h) acc = fms(acc, Li[e + h], uv[h]);
          }
          for (; e < cnt; ++e) acc = fms(acc, Li[e], U[(s0 + e) * a.m + q]);
        }
      }
      if (in) {
        const T v = col_used[q] ? zero_v<T>() : acc;
        r[q] = acc;
        u[q] = v;
        Ut[q] = v;
        const uint64_t b = entry_max_bits(v);
        cb = b > cb ? b : cb;
      }
    }
    const uint64_t gcb = cl_max(cb, x, sh, rank, ex);  // its barriers also order the row writes
    Ec = fx_entry_scale<T>(gcb, a.m);
    const T* uu = u;
    auto cw = [uu, Ec](int64_t q) -> u128 { return fx_abs2(uu[q], Ec); };
    j = cl_draw(cw, qlo, qhi - qlo, draw_u53(a.seed, t, 1, attempt), &Rfx, x, sh, rank, ex);
    if (Rfx == 0 || j < 0) {
      // the drawn row has no weight left on unpivoted columns: drop it and draw again
      if (rank == 0 && threadIdx.x == 0) {
        __stcg(d + i, 0.0);
        __threadfence();
      }
      cl_sync();
      continue;
    }
    ok = true;
    break;
  }
  cl_sync();  // every CTA is past its reads of the shared state
  if (rank != 0 || threadIdx.x != 0) return;
  double ar = 0.0, ai = 0.0;
  int32_t err = 0;
  if (ok) {
    to_d(ld_l2(r + j), ar, ai);  // written by the CTA that owns column j
    if (ar == 0.0 && ai == 0.0) {
      ok = false;
      err = kErrZeroPivot;
    }
  }
  if (!ok) {
    st->done = 1;
    st->k_done = t;
    if (err) atomicOr(&st->err, err);
    return;
  }
  a.col_used[j] = 1;
  a.row_used[i] = 1;
  a.I[t] = i;
  a.J[t] = j;
  st->i = i;
  st->j = j;
  st->a_re = ar;
  st->a_im = ai;
  st->unorm2 = fx_to_double(Rfx, Ec);
  st->cur = t;
  st->attempt = 0;
  st->redraw = 0;
  st->skip = 0;
  st->t = t + 1;
}

// ------------------------------------------------- column + row-norm update
// Per row p:
//   c_p = A(p,j) - L(p,0:t) U(0:t,j),  L(p,t) = c_p / a (FP64 division),
//   w_p = g_p - L(p,0:t) v,  d_p <- max(0, d_p - 2 Re(conj(l_p) w_p) + |l_p|^2 ||u||^2)
// with l_p the stored multiplier; L(i,t) = 1, d_i = 0, and rows pivoted earlier
// keep L(p,t) = 0 and d_p = 0.  L is read once for both sums.
//
// A CTA takes kCdRows rows at a time in two phases.  Sums: kCdLanes lanes per
// row split the s terms and the matvec's chunk partials, then combine them by
// a fixed butterfly; the s sums are in the working precision (as the residual
// row is), the chunk partials of FP32 types are summed as (hi, lo) FP32 pairs
// whose TwoSum error terms are exact (Knuth), carrying the sum to about 2^-48
// relative without the FP64 pipe, those of FP64 types in FP64.  Finish: one
// thread per row takes the FP64 division and the update, so the FP64
// instructions run with every lane of the warp busy.
constexpr int kCdLanes = 8;
constexpr int kCdRows = 64;

// Sum of chunk partials: a TwoSum pair in FP32, a plain sum in FP64.
template <typename real> struct ChunkSum;
template <> struct ChunkSum<float> {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void add(float x, float xl = 0.f) {
    const float sm = __fadd_rn(h, x);
    const float bb = __fsub_rn(sm, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(sm, bb)), __fsub_rn(x, bb));  // h + x - sm exactly
    h = sm;
    l = __fadd_rn(__fadd_rn(l, xl), e);
  }
  __device__ __forceinline__ void xor_add(int o) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
    add(h2, l2);
  }
  __device__ __forceinline__ double value() const { return (double)h + (double)l; }
};
template <> struct ChunkSum<double> {
  double h = 0.0;
  __device__ __forceinline__ void add(double x) { h += x; }
  __device__ __forceinline__ void xor_add(int o) { h += __shfl_xor_sync(0xffffffffu, h, o); }
  __device__ __forceinline__ double value() const { return h; }
};

template <typename T>
struct ColdupRow {
  typename Traits<T>::real cr, ci, wr, wi;
  double gr, gi;
};

template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cf_coldup(CauchyLaunch a) {
  using real = typename Traits<T>::real;
  __shared__ ColdupRow<T> rows[kCdRows];
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i, j = st->j;
  const double ar = st->a_re, ai = st->a_im, un2 = st->unorm2;
  const T* xv = (const T*)a.x;
  const T yj = ((const T*)a.y)[j];
  T* L = (T*)a.L;
  const T* U = (const T*)a.U;
  const T* v = (const T*)a.vproj;
  const PartT<T>* part = (const PartT<T>*)a.part;
  constexpr int RPP = kVecThreads / kCdLanes;  // rows per pass of the CTA
  constexpr int kU = 4;                        // loads issued before their (ordered) sums
  const int lane = threadIdx.x & 31, sl = lane & (kCdLanes - 1);
  const int rsub = (int)threadIdx.x / kCdLanes;
  for (int64_t tile = (int64_t)blockIdx.x * kCdRows; tile < a.n; tile += (int64_t)gridDim.x * kCdRows) {
    for (int r0 = 0; r0 < kCdRows; r0 += RPP) {
      const int rl = r0 + rsub;
      const int64_t p = tile + rl;
      const bool live = p < a.n && !a.row_used[p];
      real cr = 0, ci = 0, wr = 0, wi = 0;
      ChunkSum<real> gr, gi;
      if (live) {
        auto term = [&](T lT, T uT, T vT) {
          real lr, li, ur, ui, vr, vi;
          split(lT, lr, li);
          split(uT, ur, ui);
          split(vT, vr, vi);
          cr = lr * ur - li * ui + cr;
          ci = lr * ui + li * ur + ci;
          wr = lr * vr - li * vi + wr;
          wi = lr * vi + li * vr + wi;
        };
        int64_t s = sl;
        for (; s + (kU - 1) * kCdLanes < t; s += kU * kCdLanes) {
          T lv[kU], uv[kU], vv[kU];
#pragma unroll
          for (int h = 0; h < kU; ++h) {
            lv[h] = L[(s + h * kCdLanes) * a.n + p];
            uv[h] = U[(s + h * kCdLanes) * a.m + j];
            vv[h] = v[s + h * kCdLanes];
          }
#pragma unroll
          for (int h = 0; h < kU; ++h) term(lv[h], uv[h], vv[h]);
        }
        for (; s < t; s += kCdLanes) term(L[s * a.n + p], U[s * a.m + j], v[s]);
        int c = sl;
        for (; c + (kU - 1) * kCdLanes < a.nchunk; c += kU * kCdLanes) {
          PartT<T> g[kU];
#pragma unroll
          for (int h = 0; h < kU; ++h) g[h] = part[(int64_t)(c + h * kCdLanes) * a.n + p];
#pragma unroll
          for (int h = 0; h < kU; ++h) {
            gr.add(g[h].x);
            gi.add(g[h].y);
          }
        }
        for (; c < a.nchunk; c += kCdLanes) {
          const PartT<T> g = part[(int64_t)c * a.n + p];
          gr.add(g.x);
          gi.add(g.y);
        }
      }
#pragma unroll
      for (int o = kCdLanes / 2; o > 0; o >>= 1) {
        cr += __shfl_xor_sync(0xffffffffu, cr, o);
        ci += __shfl_xor_sync(0xffffffffu, ci, o);
        wr += __shfl_xor_sync(0xffffffffu, wr, o);
        wi += __shfl_xor_sync(0xffffffffu, wi, o);
        gr.xor_add(o);
        gi.xor_add(o);
      }
      if (sl == 0) rows[rl] = ColdupRow<T>{cr, ci, wr, wi, gr.value(), gi.value()};
    }
    __syncthreads();
    if ((int)threadIdx.x < kCdRows) {
      const int64_t p = tile + threadIdx.x;
      if (p < a.n) {
        if (a.row_used[p]) {
          if (p == i) {
            L[t * a.n + p] = one_v<T>();
            a.d[p] = 0.0;
          }
        } else {
          const ColdupRow<T> rw = rows[threadIdx.x];
          double er, ei;
          to_d(gen_entry(xv[p], yj), er, ei);
          double lr, li;
          cdiv_d(er - (double)rw.cr, ei - (double)rw.ci, ar, ai, lr, li);
          const T lT = from_d<T>(lr, li);
          L[t * a.n + p] = lT;
          to_d(lT, lr, li);
          const double w_r = rw.gr - (double)rw.wr, w_i = rw.gi - (double)rw.wi;
          // d - 2 Re(conj(l) w) + |l|^2 ||u||^2
          const double dn = a.d[p] - 2.0 * (lr * w_r + li * w_i) + (lr * lr + li * li) * un2;
          a.d[p] = dn > 0.0 ? dn : 0.0;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- CUR form
// Algorithm 2 as printed: instead of L and U, the pivot rows A(I,:) and
// columns A(:,J) are generated again and the core inverse Uc = A(I,J)^{-1}
// (FP64) is updated by block inversion (Eq. block-inverse-update).  With
// t pivots so far and the row i of this step:
//   b^T = A(i,J) Uc,   r = A(i,:) - b^T A(I,:)                  (residual row)
//   e = Uc A(I,j),     c = A(:,j) - A(:,J) e, l = c / a           (residual column)
//   g = A conj(u),     w = g - A(:,J) (Uc g(I))                   (residual times conj(u))
//   Uc <- [[Uc + e b^T / a, -e / a], [-b^T / a, 1 / a]],  a = r_j  (the block inverse)
// The entries these kernels generate, and their sums, are FP64 for every data
// type: FP32 points are widened first (their difference is exact in FP64), so
// the core inverts the matrix of the given points to FP64 accuracy instead of
// its FP32-rounded entries, whose error the inverse would amplify by the
// condition number of A(I,J).
__device__ __forceinline__ cf64 gen_d(float x, float y) { return cf64{1.0 / ((double)x - (double)y), 0.0}; }
__device__ __forceinline__ cf64 gen_d(double x, double y) { return cf64{gen_entry(x, y), 0.0}; }
__device__ __forceinline__ cf64 gen_d(cf32 x, cf32 y) {
  return gen_entry(cf64{(double)x.re, (double)x.im}, cf64{(double)y.re, (double)y.im});
}
__device__ __forceinline__ cf64 gen_d(cf64 x, cf64 y) { return gen_entry(x, y); }
__device__ __forceinline__ void cmac(cf64& acc, cf64 a, cf64 b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}

// b_s = sum_p A(i, J_p) Uc(p, s), one thread per s
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cur_b(CauchyLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  const T xi = x[i];
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < t; s += (int64_t)gridDim.x * blockDim.x) {
    cf64 acc{0.0, 0.0};
    for (int64_t p = 0; p < t; ++p) cmac(acc, gen_d(xi, y[a.J[p]]), a.core[p * a.k + s]);
    a.vb[s] = acc;
  }
}

// r_q = A(i,q) - sum_s b_s A(I_s, q)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cur_row(CauchyLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  T* r = (T*)a.rhat;
  const T xi = x[i];
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.m; q += (int64_t)gridDim.x * blockDim.x) {
    const T yq = y[q];
    cf64 acc = gen_d(xi, yq);
    for (int64_t s = 0; s < t; ++s) {
      const cf64 bs = a.vb[s], v = gen_d(x[a.I[s]], yq);
      acc.re -= bs.re * v.re - bs.im * v.im;
      acc.im -= bs.re * v.im + bs.im * v.re;
    }
    r[q] = from_d<T>(acc.re, acc.im);
  }
}

// e_p = sum_s Uc(p, s) A(I_s, j), one warp per p (lanes over s)
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cur_e(CauchyLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, j = st->j;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  const int lane = threadIdx.x & 31;
  const T yj = y[j];
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < t;
       p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    cf64 acc{0.0, 0.0};
    for (int64_t s = lane; s < t; s += 32) cmac(acc, a.core[p * a.k + s], gen_d(x[a.I[s]], yj));
    for (int o = 16; o > 0; o >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (lane == 0) a.ve[p] = acc;
  }
}

// c_p = A(p,j) - sum_s A(p, J_s) e_s ; L-column multipliers l = c / a (FP64
// division), l_i = 1, 0 on the rows pivoted before
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cur_col(CauchyLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i, j = st->j;
  const double ar = st->a_re, ai = st->a_im;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  T* lc = (T*)a.lcol;
  const T yj = y[j];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    if (a.row_used[p]) {
      lc[p] = p == i ? one_v<T>() : zero_v<T>();
      continue;
    }
    const T xp = x[p];
    cf64 acc = gen_d(xp, yj);
    for (int64_t s = 0; s < t; ++s) {
      const cf64 es = a.ve[s], v = gen_d(xp, y[a.J[s]]);
      acc.re -= v.re * es.re - v.im * es.im;
      acc.im -= v.re * es.im + v.im * es.re;
    }
    double lr, li;
    cdiv_d(acc.re, acc.im, ar, ai, lr, li);
    lc[p] = from_d<T>(lr, li);
  }
}

// g(I_s) from the matvec's chunk partials (FP64 sum), one thread per s
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cur_gI(CauchyLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur;
  const PartT<T>* part = (const PartT<T>*)a.part;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < t; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = a.I[s];
    double gr = 0.0, gi = 0.0;
    for (int c = 0; c < a.nchunk; ++c) {
      const PartT<T> g = part[(int64_t)c * a.n + row];
      gr += (double)g.x;
      gi += (double)g.y;
    }
    a.vg[s] = cf64{gr, gi};
  }
}

// h_p = sum_s Uc(p, s) g(I_s), one warp per p
__global__ void __launch_bounds__(kVecThreads) k_cur_h(CauchyLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur;
  const int lane = threadIdx.x & 31;
  for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < t;
       p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    cf64 acc{0.0, 0.0};
    for (int64_t s = lane; s < t; s += 32) cmac(acc, a.core[p * a.k + s], a.vg[s]);
    for (int o = 16; o > 0; o >>= 1) {
      acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
      acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
    }
    if (lane == 0) a.vh[p] = acc;
  }
}

// w_p = g_p - sum_s A(p, J_s) h_s ; d update of Sec. 4.1
template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_cur_dupdate(CauchyLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur, i = st->i;
  const double un2 = st->unorm2;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  const T* lc = (const T*)a.lcol;
  const PartT<T>* part = (const PartT<T>*)a.part;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    if (a.row_used[p]) {
      if (p == i) a.d[p] = 0.0;
      continue;
    }
    double wr = 0.0, wi = 0.0;
    for (int c = 0; c < a.nchunk; ++c) {
      const PartT<T> g = part[(int64_t)c * a.n + p];
      wr += (double)g.x;
      wi += (double)g.y;
    }
    const T xp = x[p];
    for (int64_t s = 0; s < t; ++s) {
      const cf64 hs = a.vh[s], v = gen_d(xp, y[a.J[s]]);
      wr -= v.re * hs.re - v.im * hs.im;
      wi -= v.re * hs.im + v.im * hs.re;
    }
    double lr, li;
    to_d(lc[p], lr, li);
    const double dn = a.d[p] - 2.0 * (lr * wr + li * wi) + (lr * lr + li * li) * un2;
    a.d[p] = dn > 0.0 ? dn : 0.0;
  }
}

// Uc <- [[Uc + e b^T / a, -e / a], [-b^T / a, 1 / a]] (in place, (t+1)^2 entries)
__global__ void __launch_bounds__(kVecThreads) k_cur_core(CauchyLaunch a) {
  const JobState* st = a.st;
  if (st->done || st->skip) return;
  const int64_t t = st->cur;
  double sr, si;  // 1 / a
  {
    const double ar = st->a_re, ai = st->a_im;
    cdiv_d(1.0, 0.0, ar, ai, sr, si);
  }
  const int64_t t1 = t + 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < t1 * t1; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / t1, s = e - p * t1;
    cf64 v;
    if (p < t && s < t) {
      const cf64 ep = a.ve[p], bs = a.vb[s];
      const double pr = ep.re * bs.re - ep.im * bs.im, pi = ep.re * bs.im + ep.im * bs.re;
      v = a.core[p * a.k + s];
      v.re += pr * sr - pi * si;
      v.im += pr * si + pi * sr;
    } else if (p < t) {
      const cf64 ep = a.ve[p];
      v = cf64{-(ep.re * sr - ep.im * si), -(ep.re * si + ep.im * sr)};
    } else if (s < t) {
      const cf64 bs = a.vb[s];
      v = cf64{-(bs.re * sr - bs.im * si), -(bs.re * si + bs.im * sr)};
    } else {
      v = cf64{sr, si};
    }
    a.core[p * a.k + s] = v;
  }
}

__global__ void __launch_bounds__(kSmpThreads) k_cf_finish(CauchyLaunch a) {
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

inline unsigned grid_for(int64_t work, int threads, int num_sms, int per_sm) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

template <typename T>
cudaError_t init_t(const CauchyLaunch& a, cudaStream_t s, HotTimer* tm) {
  if (a.n == 0 || a.m == 0) return cudaGetLastError();
  const dim3 grid((unsigned)((a.n + kMvThreads * kMvRows - 1) / (kMvThreads * kMvRows)), (unsigned)a.nchunk);
  k_cf_matvec<T, true><<<grid, kMvThreads, 0, s>>>(a);
  k_cf_norm_reduce<T><<<grid_for(a.n, kVecThreads, a.num_sms, 8), kVecThreads, 0, s>>>(a);
  tm->all_launches += 2;
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_t(const CauchyLaunch& a, cudaStream_t s, int64_t steps, HotTimer* tm) {
  const dim3 mv_grid((unsigned)((a.n + kMvThreads * kMvRows - 1) / (kMvThreads * kMvRows)), (unsigned)a.nchunk);
  const unsigned gm = grid_for(a.m, kVecThreads, a.num_sms, 8);
  const unsigned gcd = grid_for((a.n + kCdRows - 1) / kCdRows * kVecThreads, kVecThreads, a.num_sms, 8);
  for (int64_t q = 0; q < steps; ++q) {
    if (a.mode == RPLU_PIVOT_RANDOM) {
      k_cf_pivot_cl<T><<<kCl, kClThreads, 0, s>>>(a);
      tm->all_launches += 1;
    } else {
      k_cf_sample_row<<<1, kSmpThreads, 0, s>>>(a);
      k_cf_row<T><<<gm, kVecThreads, 0, s>>>(a);
      k_cf_sample_col<T><<<1, kSmpThreads, 0, s>>>(a);
      tm->all_launches += 3;
    }
    tm->begin();
    k_cf_matvec<T, false><<<mv_grid, kMvThreads, 0, s>>>(a);
    tm->end();
    k_cf_coldup<T><<<gcd, kVecThreads, 0, s>>>(a);
    tm->all_launches += 2;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t cur_run_t(const CauchyLaunch& a, cudaStream_t s, int64_t steps, HotTimer* tm) {
  const dim3 mv_grid((unsigned)((a.n + kMvThreads * kMvRows - 1) / (kMvThreads * kMvRows)), (unsigned)a.nchunk);
  const unsigned gn = grid_for(a.n, kVecThreads, a.num_sms, 8);
  const unsigned gm = grid_for(a.m, kVecThreads, a.num_sms, 8);
  const unsigned gk = grid_for(a.k, kVecThreads, a.num_sms, 8);
  const unsigned gw = grid_for(a.k * 32, kVecThreads, a.num_sms, 8);
  const unsigned gkk = grid_for(a.k * a.k, kVecThreads, a.num_sms, 8);
  for (int64_t q = 0; q < steps; ++q) {
    k_cf_sample_row<<<1, kSmpThreads, 0, s>>>(a);
    k_cur_b<T><<<gk, kVecThreads, 0, s>>>(a);
    k_cur_row<T><<<gm, kVecThreads, 0, s>>>(a);
    k_cf_sample_col<T><<<1, kSmpThreads, 0, s>>>(a);
    k_cur_e<T><<<gw, kVecThreads, 0, s>>>(a);
    k_cur_col<T><<<gn, kVecThreads, 0, s>>>(a);
    tm->begin();
    k_cf_matvec<T, false><<<mv_grid, kMvThreads, 0, s>>>(a);
    tm->end();
    k_cur_gI<T><<<gk, kVecThreads, 0, s>>>(a);
    k_cur_h<<<gw, kVecThreads, 0, s>>>(a);
    k_cur_dupdate<T><<<gn, kVecThreads, 0, s>>>(a);
    k_cur_core<<<gkk, kVecThreads, 0, s>>>(a);
    tm->all_launches += 11;
  }
  return cudaGetLastError();
}

}  // namespace

// The core leaves in FP64 for every data type (float64 for real data,
// complex128 for complex data): it is an inverse, with the condition number of
// A(I,J), which FP32 could not carry.
template <typename TO>
__global__ void k_core_out(const cf64* core, int64_t k, int64_t kd, TO* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / k, q = e - p * k;
    out[e] = (p < kd && q < kd) ? from_d<TO>(core[e].re, core[e].im) : zero_v<TO>();
  }
}

cudaError_t cauchy_core_out(int32_t dtype, const cf64* core, int64_t k, int64_t kd, void* out, int num_sms,
                            cudaStream_t s) {
  const unsigned g = grid_for(k * k, kVecThreads, num_sms, 8);
  switch (dtype) {
    case RPLU_F32:
    case RPLU_F64: k_core_out<double><<<g, kVecThreads, 0, s>>>(core, k, kd, (double*)out); break;
    case RPLU_C64:
    case RPLU_C128: k_core_out<cf64><<<g, kVecThreads, 0, s>>>(core, k, kd, (cf64*)out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t cauchy_cur_run(int32_t dtype, const CauchyLaunch& a, cudaStream_t s, int64_t steps, HotTimer* tm) {
  switch (dtype) {
    case RPLU_F32: return cur_run_t<float>(a, s, steps, tm);
    case RPLU_F64: return cur_run_t<double>(a, s, steps, tm);
    case RPLU_C64: return cur_run_t<cf32>(a, s, steps, tm);
    case RPLU_C128: return cur_run_t<cf64>(a, s, steps, tm);
    default: return cudaErrorInvalidValue;
  }
}

// Matvec CTAs resident per SM for a data type (the registers bound it), from
// the occupancy calculator of the current device; 0 when it cannot say.
template <typename T>
int mv_ctas_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cf_matvec<T, false>, kMvThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

// Column chunks of the matvec grid (row tiles x chunks CTAs): about 8 CTAs per
// SM in all, rounded down to whole waves of resident CTAs.  Rounding up
// instead (1220 CTAs for 20000 rows on 152 SMs holding 4 each: two full waves
// and a third of 4 CTAs) leaves the GPU nearly idle for a whole CTA time.
int32_t cauchy_chunks(int64_t n, int64_t m, int32_t dtype, int32_t num_sms) {
  const int64_t tiles = std::max<int64_t>(1, (n + kMvThreads * kMvRows - 1) / (kMvThreads * kMvRows));
  const int nb = dtype == RPLU_F32 ? mv_ctas_per_sm<float>() : dtype == RPLU_F64 ? mv_ctas_per_sm<double>()
                 : dtype == RPLU_C64 ? mv_ctas_per_sm<cf32>() : mv_ctas_per_sm<cf64>();
  const int64_t target = (int64_t)num_sms * 8;
  int64_t c;
  if (nb > 0) {
    const int64_t slots = (int64_t)num_sms * nb;  // one wave
    const int64_t waves = (target + slots - 1) / slots;
    c = waves * slots / tiles;
  } else {
    c = (target + tiles - 1) / tiles;
  }
  const int64_t cmax = (m + 63) / 64;
  if (c > cmax) c = cmax;
  if (c > 65535) c = 65535;
  if (c < 1) c = 1;
  return (int32_t)c;
}

cudaError_t cauchy_init(int32_t dtype, const CauchyLaunch& a, cudaStream_t s, HotTimer* tm) {
  switch (dtype) {
    case RPLU_F32: return init_t<float>(a, s, tm);
    case RPLU_F64: return init_t<double>(a, s, tm);
    case RPLU_C64: return init_t<cf32>(a, s, tm);
    case RPLU_C128: return init_t<cf64>(a, s, tm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t cauchy_run(int32_t dtype, const CauchyLaunch& a, cudaStream_t s, int64_t steps, HotTimer* tm) {
  switch (dtype) {
    case RPLU_F32: return run_t<float>(a, s, steps, tm);
    case RPLU_F64: return run_t<double>(a, s, steps, tm);
    case RPLU_C64: return run_t<cf32>(a, s, steps, tm);
    case RPLU_C128: return run_t<cf64>(a, s, steps, tm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t cauchy_finish(const CauchyLaunch& a, cudaStream_t s, HotTimer* tm) {
  k_cf_finish<<<1, kSmpThreads, 0, s>>>(a);
  tm->all_launches += 1;
  return cudaGetLastError();
}

}  // namespace rplu
