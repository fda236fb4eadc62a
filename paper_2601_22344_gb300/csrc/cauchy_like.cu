// RPLU of Cauchy-like matrices through their generators (Sec. 5.1): A_pq =
// sum_l G[p,l] B[l,q] / (x_p - y_q) (Eq. cauchy-like).  Every residual is
// Cauchy-like with generators updated by Eqs. generator_update_g / _b, so the
// residual is never stored and its entries are generated from x, y, G, B.
// Unlike the matrix-free LU form (cauchy.cu), the squared row norms are
// recomputed exactly from the generated residual at every step (Algorithm 3
// samples with bounds and rejection instead), so they carry no drift.
//
// Per step:
//   k_cl_norms       (grid)   partial sums of |S_pq|^2 over column chunks
//   k_cl_norm_reduce (grid)   d_p = sum of the partials (FP64, chunk order)
//   k_cl_sample      (1 CTA)  T = sum d, stop test, row draw by d, pivot row
//                             r = S(i,:), column draw by |r_q|^2 (pivoted
//                             columns masked), U(t,:) = r, saves G(i,:), B(:,j)
//   k_cl_update      (grid)   c_p = S(p,j); L(:,t) = c/a (L(i,t) = 1,
//                             L(I_prev,t) = 0); G <- G - L(:,t) G(i,:);
//                             B <- B - B(:,j) (r / a); G(i,:) = B(:,j) = 0
#include <type_traits>

#include "cauchy_like.cuh"
#include "common.cuh"
#include "kernels.h"
#include "packed.cuh"
#include "sampler.cuh"

namespace rplu {
namespace {

constexpr int kNThreads = 256;  // norm kernel CTA size; also the shared tile width
constexpr int kNRows = 4;       // rows per norm thread
constexpr int kSThreads = 1024;
constexpr int kUThreads = 256;

// ------------------------------------------------------------- row norms
// d_p = sum_q |S_pq|^2 over the column chunk blockIdx.y: per entry the
// generator product (P multiply-adds) and |s|^2 / |x_p - y_q|^2 with a fast
// reciprocal; squares summed in the working precision per 256-column tile,
// tiles summed in FP64.  FP32 data (real and complex) take the same
// arithmetic two rows at a time in packed f32x2 instructions; the column's
// values are staged duplicated ({v, v}) so that they feed a pair directly.
struct alignas(8) Dup { float2 v; };

// Whether a row-norm pass runs: every step of the exact-norm form; under the
// bound-based draw only the passes forced by the host (the initial and final
// exact totals) and those of a step whose proposals were all rejected.
__device__ __forceinline__ bool norms_wanted(const CauchyLikeLaunch& a) {
  if (a.gate == kGateForced) return true;
  if (a.st->done) return false;
  return a.gate == kGateNone || a.st->fallback != 0;
}

template <typename T, int P>
__global__ void __launch_bounds__(kNThreads) k_cl_norms(CauchyLikeLaunch a) {
  using real = typename Traits<T>::real;
  if (!norms_wanted(a)) return;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  const T* G = (const T*)a.G;
  const T* Bm = (const T*)a.B;
  const int64_t row0 = (int64_t)blockIdx.x * (kNThreads * kNRows) + threadIdx.x;
  const int64_t chunk = (a.m + a.nchunk - 1) / a.nchunk;
  const int64_t q0 = (int64_t)blockIdx.y * chunk;
  const int64_t q1 = min(a.m, q0 + chunk);
  double acc[kNRows];
#pragma unroll
  for (int r = 0; r < kNRows; ++r) acc[r] = 0.0;
  if constexpr (std::is_same<T, float>::value || std::is_same<T, cf32>::value) {
    constexpr bool C = std::is_same<T, cf32>::value;
    constexpr int NP = kNRows / 2;  // row pairs per thread
    // per column: {y_re}, {y_im}, then per generator l: {b_re}, {b_im}, {-b_im};
    // with p = 1, |g_p b_q|^2 = |g_p|^2 |b_q|^2, so only {|b_q|^2} is staged
    // and |g_p|^2 multiplies each row's tile sum
    constexpr int NV = P == 1 ? (C ? 3 : 2) : (C ? 2 + 3 * P : 1 + P);
    __shared__ float2 tv[NV][kNThreads];
    float2 xr2[NP], xi2[NP], gr2[NP][P], gi2[NP][P];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      float xv[2][2], gv[2][P][2];
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t p = row0 + (int64_t)(2 * h + e) * kNThreads;
        const int64_t pc = p < a.n ? p : a.n - 1;
        const T xp = x[pc];
        xv[e][0] = re_of(xp);
        xv[e][1] = im_of(xp);
#pragma unroll
        for (int l = 0; l < P; ++l) {
          const T gp = p < a.n ? G[pc * P + l] : zero_v<T>();
          gv[e][l][0] = re_of(gp);
          gv[e][l][1] = im_of(gp);
        }
      }
      xr2[h] = make_float2(xv[0][0], xv[1][0]);
      xi2[h] = make_float2(xv[0][1], xv[1][1]);
#pragma unroll
      for (int l = 0; l < P; ++l) {
        gr2[h][l] = make_float2(gv[0][l][0], gv[1][l][0]);
        gi2[h][l] = make_float2(gv[0][l][1], gv[1][l][1]);
      }
    }
    for (int64_t qt = q0; qt < q1; qt += kNThreads) {
      const int cnt = (int)min((int64_t)kNThreads, q1 - qt);
      __syncthreads();
      if ((int)threadIdx.x < cnt) {
        const int64_t q = qt + threadIdx.x;
        const T yq = y[q];
        tv[0][threadIdx.x] = f2_splat(re_of(yq));
        if constexpr (C) tv[1][threadIdx.x] = f2_splat(im_of(yq));
        if constexpr (P == 1) {
          const T b = Bm[q];
          const float br = re_of(b), bi = im_of(b);
          tv[C ? 2 : 1][threadIdx.x] = f2_splat(fmaf(br, br, bi * bi));
        }
#pragma unroll
        for (int l = 0; l < (P == 1 ? 0 : P); ++l) {
          const T b = Bm[(int64_t)l * a.m + q];
          if constexpr (C) {
            tv[2 + 3 * l][threadIdx.x] = f2_splat(re_of(b));
            tv[3 + 3 * l][threadIdx.x] = f2_splat(im_of(b));
            tv[4 + 3 * l][threadIdx.x] = f2_splat(-im_of(b));
          } else {
            tv[1 + l][threadIdx.x] = f2_splat(re_of(b));
          }
        }
      }
      __syncthreads();
      float2 tile[NP];
#pragma unroll
      for (int h = 0; h < NP; ++h) tile[h] = make_float2(0.f, 0.f);
      for (int qq = 0; qq < cnt; ++qq) {
        const float2 yr = tv[0][qq];
#pragma unroll
        for (int h = 0; h < NP; ++h) {
          if constexpr (P == 1) {
            // |b_q|^2 / |x_p - y_q|^2, two rows at once
            float2 z2;
            if constexpr (C) {
              const float2 zr = f2_sub(xr2[h], yr), zi = f2_sub(xi2[h], tv[1][qq]);
              z2 = f2_fma(zr, zr, f2_mul(zi, zi));
            } else {
              const float2 z = f2_sub(xr2[h], yr);
              z2 = f2_mul(z, z);
            }
            const float2 inv = make_float2(rcp_fast(z2.x), rcp_fast(z2.y));
            tile[h] = f2_fma(tv[C ? 2 : 1][qq], inv, tile[h]);
          } else if constexpr (C) {
            const float2 yi = tv[1][qq];
            // s = sum_l g_l b_l (complex), two rows at once
            float2 sr = f2_mul(gr2[h][0], tv[2][qq]);
            sr = f2_fma(gi2[h][0], tv[4][qq], sr);
            float2 si = f2_mul(gr2[h][0], tv[3][qq]);
            si = f2_fma(gi2[h][0], tv[2][qq], si);
#pragma unroll
            for (int l = 1; l < P; ++l) {
              sr = f2_fma(gr2[h][l], tv[2 + 3 * l][qq], sr);
              sr = f2_fma(gi2[h][l], tv[4 + 3 * l][qq], sr);
              si = f2_fma(gr2[h][l], tv[3 + 3 * l][qq], si);
              si = f2_fma(gi2[h][l], tv[2 + 3 * l][qq], si);
            }
            const float2 zr = f2_sub(xr2[h], yr), zi = f2_sub(xi2[h], yi);
            const float2 s2 = f2_fma(sr, sr, f2_mul(si, si));
            const float2 z2 = f2_fma(zr, zr, f2_mul(zi, zi));
            const float2 inv = make_float2(rcp_fast(z2.x), rcp_fast(z2.y));
            tile[h] = f2_fma(s2, inv, tile[h]);
          } else {
            float2 sv = f2_mul(gr2[h][0], tv[1][qq]);
#pragma unroll
            for (int l = 1; l < P; ++l) sv = f2_fma(gr2[h][l], tv[1 + l][qq], sv);
            const float2 z = f2_sub(xr2[h], yr);
            const float2 ev = f2_mul(sv, make_float2(rcp_fast(z.x), rcp_fast(z.y)));
            tile[h] = f2_fma(ev, ev, tile[h]);
          }
        }
      }
#pragma unroll
      for (int h = 0; h < NP; ++h) {
        if constexpr (P == 1) {
          // |g_p|^2 times the tile's sum of |b_q|^2 / |z|^2
          const float g0 = fmaf(gr2[h][0].x, gr2[h][0].x, gi2[h][0].x * gi2[h][0].x);
          const float g1 = fmaf(gr2[h][0].y, gr2[h][0].y, gi2[h][0].y * gi2[h][0].y);
          acc[2 * h] += (double)g0 * (double)tile[h].x;
          acc[2 * h + 1] += (double)g1 * (double)tile[h].y;
        } else {
          acc[2 * h] += (double)tile[h].x;
          acc[2 * h + 1] += (double)tile[h].y;
        }
      }
    }
  } else {
    __shared__ T ty[kNThreads];
    __shared__ T tb[P][kNThreads];
    T xr[kNRows];
    T g[kNRows][P];
#pragma unroll
    for (int r = 0; r < kNRows; ++r) {
      const int64_t p = row0 + (int64_t)r * kNThreads;
      const int64_t pc = p < a.n ? p : a.n - 1;
      xr[r] = x[pc];
#pragma unroll
      for (int l = 0; l < P; ++l) g[r][l] = p < a.n ? G[pc * P + l] : zero_v<T>();
    }
    for (int64_t qt = q0; qt < q1; qt += kNThreads) {
      const int cnt = (int)min((int64_t)kNThreads, q1 - qt);
      __syncthreads();
      if ((int)threadIdx.x < cnt) {
        const int64_t q = qt + threadIdx.x;
        ty[threadIdx.x] = y[q];
#pragma unroll
        for (int l = 0; l < P; ++l) tb[l][threadIdx.x] = Bm[(int64_t)l * a.m + q];
      }
      __syncthreads();
      real tile[kNRows];
#pragma unroll
      for (int r = 0; r < kNRows; ++r) tile[r] = 0;
      for (int qq = 0; qq < cnt; ++qq) {
        const T yv = ty[qq];
        T bv[P];
#pragma unroll
        for (int l = 0; l < P; ++l) bv[l] = tb[l][qq];
#pragma unroll
        for (int r = 0; r < kNRows; ++r) {
          T sv = mul_v(g[r][0], bv[0]);
#pragma unroll
          for (int l = 1; l < P; ++l) sv = add_v(sv, mul_v(g[r][l], bv[l]));
          const real zr = re_of(xr[r]) - re_of(yv), zi = im_of(xr[r]) - im_of(yv);
          const real sr = re_of(sv), si = im_of(sv);
          tile[r] += (sr * sr + si * si) * rcp_fast(zr * zr + zi * zi);
        }
      }
#pragma unroll
      for (int r = 0; r < kNRows; ++r) acc[r] += (double)tile[r];
    }
  }
#pragma unroll
  for (int r = 0; r < kNRows; ++r) {
    const int64_t p = row0 + (int64_t)r * kNThreads;
    if (p < a.n) a.part[(int64_t)blockIdx.y * a.n + p] = acc[r];
  }
}

__global__ void __launch_bounds__(kUThreads) k_cl_norm_reduce(CauchyLikeLaunch a) {
  if (!norms_wanted(a)) return;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < a.nchunk; ++c) s += a.part[(int64_t)c * a.n + p];
    a.d[p] = a.row_used[p] ? 0.0 : s;
  }
}

// ---------------------------------------------------------------- sample
template <typename T, int P>
__global__ void __launch_bounds__(kSThreads) k_cl_sample(CauchyLikeLaunch a) {
  __shared__ FxScratch sh;
  JobState* st = a.st;
  if (st->done) return;
  const int64_t t = st->t;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  const T* G = (const T*)a.G;
  const T* Bm = (const T*)a.B;
  T* r = (T*)a.r;
  T* urow = (T*)a.U + t * a.m;
  double* d = a.d;
  const uint8_t* col_used = a.col_used;
  uint64_t mb = max_bits_f64(d, a.n);
  mb = block_max_u64(mb, sh);
  const int Er = fx_scale_f64(mb, a.n);
  auto dw = [d, Er](int64_t p) -> u128 { return fx_f64(d[p], Er); };
  int64_t i = -1, j = -1;
  bool ok = false;
  int32_t err = 0;
  for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
    u128 Tfx;
    if (a.mode == RPLU_PIVOT_RANDOM) {
      i = fx_block_draw(dw, a.n, draw_u53(a.seed, t, 0, attempt), true, &Tfx, sh);
    } else {
      (void)fx_block_draw(dw, a.n, 0, false, &Tfx, sh);
      if (a.mode == RPLU_PIVOT_C2) i = fx_block_argmax([d](int64_t p) -> uint64_t { return fx_bits64(d[p]); }, a.n, sh);
      else i = a.gI[t];
    }
    const double T_ = fx_to_double(Tfx, Er);
    if (attempt == 0) {
      const double T0 = (t == 0) ? T_ : st->T0;
      if (threadIdx.x == 0) {
        a.T_hist[t] = T_;
        if (t == 0) st->T0 = T_;
      }
      if (!(T_ > 0.0) || (a.tol > 0.0 && T_ <= a.tol * a.tol * T0)) break;
    } else if (!(T_ > 0.0)) {
      break;
    }
    if (a.mode == RPLU_PIVOT_GIVEN && (i < 0 || i >= a.n || a.row_used[i])) {
      err = kErrBadGiven;
      break;
    }
    if (i < 0) break;
    // pivot row r = S(i,:) from the generators, pivoted columns masked
    T gi[P];
#pragma unroll
    for (int l = 0; l < P; ++l) gi[l] = G[i * P + l];
    const T xi = x[i];
    uint64_t cb = 0;
    for (int64_t q = threadIdx.x; q < a.m; q += blockDim.x) {
      T bq[P];
#pragma unroll
      for (int l = 0; l < P; ++l) bq[l] = Bm[(int64_t)l * a.m + q];
      T v = col_used[q] ? zero_v<T>() : entry_gen<T, P>(gi, bq, xi, y[q]);
      r[q] = v;
      urow[q] = v;
      const uint64_t b = entry_max_bits(v);
      cb = b > cb ? b : cb;
    }
    cb = block_max_u64(cb, sh);  // also orders the row writes before the reads below
    const int Ec = fx_entry_scale<T>(cb, a.m);
    const T* rr = r;
    auto cw = [rr, Ec](int64_t q) -> u128 { return fx_abs2(rr[q], Ec); };
    u128 Rfx = 1;
    if (a.mode == RPLU_PIVOT_RANDOM) {
      j = fx_block_draw(cw, a.m, draw_u53(a.seed, t, 1, attempt), true, &Rfx, sh);
    } else if (a.mode == RPLU_PIVOT_C2) {
      (void)fx_block_draw(cw, a.m, 0, false, &Rfx, sh);
      j = fx_block_argmax(cw, a.m, sh);
    } else {
      j = a.gJ[t];
      if (j < 0 || j >= a.m || col_used[j]) {
        err = kErrBadGiven;
        break;
      }
    }
    if (Rfx == 0 || j < 0) {
      if (threadIdx.x == 0) d[i] = 0.0;
      __syncthreads();
      continue;
    }
    ok = true;
    break;
  }
  double ar = 0.0, ai = 0.0;
  if (ok) {
    to_d(r[j], ar, ai);
    if (ar == 0.0 && ai == 0.0) {
      ok = false;
      err = kErrZeroPivot;
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) {
      st->done = 1;
      st->k_done = t;
      if (err) atomicOr(&st->err, err);
    }
    return;
  }
  __syncthreads();
  if (threadIdx.x < P) {
    ((T*)a.gi)[threadIdx.x] = G[i * P + threadIdx.x];
    ((T*)a.bj)[threadIdx.x] = Bm[(int64_t)threadIdx.x * a.m + j];
  }
  if (threadIdx.x == 0) {
    a.col_used[j] = 1;
    a.row_used[i] = 1;
    a.I[t] = i;
    a.J[t] = j;
    st->i = i;
    st->j = j;
    st->a_re = ar;
    st->a_im = ai;
    st->cur = t;
    st->t = t + 1;
  }
}

// ---------------------------------------------------------------- update
// Threads [0, n): pivot column entry, L(:,t) and G; threads [n, n + m): B.
template <typename T, int P>
__global__ void __launch_bounds__(kUThreads) k_cl_update(CauchyLikeLaunch a) {
  JobState* st = a.st;
  if (st->done) return;
  const int64_t t = st->cur, i = st->i, j = st->j;
  const double ar = st->a_re, ai = st->a_im;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  T* G = (T*)a.G;
  T* Bm = (T*)a.B;
  const T* r = (const T*)a.r;
  T gi[P], bj[P];
#pragma unroll
  for (int l = 0; l < P; ++l) {
    gi[l] = ((const T*)a.gi)[l];
    bj[l] = ((const T*)a.bj)[l];
  }
  T* Lt = (T*)a.L + t * a.n;
  const int64_t total = a.n + a.m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < a.n) {
      const int64_t p = e;
      if (p == i) {
        Lt[p] = one_v<T>();
#pragma unroll
        for (int l = 0; l < P; ++l) G[p * P + l] = zero_v<T>();
      } else if (a.row_used[p]) {
        Lt[p] = zero_v<T>();
      } else {
        T gp[P];
#pragma unroll
        for (int l = 0; l < P; ++l) gp[l] = G[p * P + l];
        const T c = entry_gen<T, P>(gp, bj, x[p], y[j]);
        double cr, ci, lr, li;
        to_d(c, cr, ci);
        cdiv_d(cr, ci, ar, ai, lr, li);
        const T lp = from_d<T>(lr, li);
        Lt[p] = lp;
#pragma unroll
        for (int l = 0; l < P; ++l) G[p * P + l] = sub_v(gp[l], mul_v(lp, gi[l]));
      }
    } else {
      const int64_t q = e - a.n;
      if (q == j) {
#pragma unroll
        for (int l = 0; l < P; ++l) Bm[(int64_t)l * a.m + q] = zero_v<T>();
      } else {
        double rr_, ri_, ur, ui;
        to_d(r[q], rr_, ri_);
        cdiv_d(rr_, ri_, ar, ai, ur, ui);
        const T uq = from_d<T>(ur, ui);
#pragma unroll
        for (int l = 0; l < P; ++l) Bm[(int64_t)l * a.m + q] = sub_v(Bm[(int64_t)l * a.m + q], mul_v(bj[l], uq));
      }
    }
  }
}

__global__ void k_cl_finish(CauchyLikeLaunch a) {
  __shared__ FxScratch sh;
  JobState* st = a.st;
  const double T_ = fx_total_f64(a.d, a.n, sh);
  if (threadIdx.x == 0) {
    if (!st->done) {
      st->done = 1;
      st->k_done = a.k;
    }
    a.T_hist[st->k_done] = T_;
    if (a.k == 0) st->T0 = T_;
  }
}

template <typename T, int P>
cudaError_t run_tp(const CauchyLikeLaunch& a, cudaStream_t s, HotTimer* tm) {
  const dim3 ng((unsigned)((a.n + kNThreads * kNRows - 1) / (kNThreads * kNRows)), (unsigned)a.nchunk);
  const unsigned rg = (unsigned)std::min<int64_t>((a.n + kUThreads - 1) / kUThreads, (int64_t)a.num_sms * 8);
  const unsigned ug = (unsigned)std::min<int64_t>((a.n + a.m + kUThreads - 1) / kUThreads, (int64_t)a.num_sms * 8);
  for (int64_t t = 0; t <= a.k; ++t) {
    tm->begin();
    k_cl_norms<T, P><<<ng, kNThreads, 0, s>>>(a);
    tm->end();
    k_cl_norm_reduce<<<std::max(rg, 1u), kUThreads, 0, s>>>(a);
    tm->all_launches += 2;
    if (t == a.k) break;
    k_cl_sample<T, P><<<1, kSThreads, 0, s>>>(a);
    k_cl_update<T, P><<<std::max(ug, 1u), kUThreads, 0, s>>>(a);
    tm->all_launches += 2;
  }
  k_cl_finish<<<1, 1024, 0, s>>>(a);
  tm->all_launches += 1;
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_t(const CauchyLikeLaunch& a, cudaStream_t s, HotTimer* tm) {
  switch (a.p) {
    case 1: return run_tp<T, 1>(a, s, tm);
    case 2: return run_tp<T, 2>(a, s, tm);
    case 3: return run_tp<T, 3>(a, s, tm);
    case 4: return run_tp<T, 4>(a, s, tm);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int P>
void launch_norms_tp(const CauchyLikeLaunch& a, cudaStream_t s) {
  const dim3 ng((unsigned)((a.n + kNThreads * kNRows - 1) / (kNThreads * kNRows)), (unsigned)a.nchunk);
  const unsigned rg = (unsigned)std::min<int64_t>((a.n + kUThreads - 1) / kUThreads, (int64_t)a.num_sms * 8);
  k_cl_norms<T, P><<<ng, kNThreads, 0, s>>>(a);
  k_cl_norm_reduce<<<std::max(rg, 1u), kUThreads, 0, s>>>(a);
}

template <typename T, int P>
void launch_update_tp(const CauchyLikeLaunch& a, cudaStream_t s) {
  const unsigned ug = (unsigned)std::min<int64_t>((a.n + a.m + kUThreads - 1) / kUThreads, (int64_t)a.num_sms * 8);
  k_cl_update<T, P><<<std::max(ug, 1u), kUThreads, 0, s>>>(a);
}

template <typename T>
cudaError_t launch_t(int which, const CauchyLikeLaunch& a, cudaStream_t s) {
  switch (a.p) {
#define RPLU_CL_P(P)                                          \
    case P:                                                   \
      if (which == 0) launch_norms_tp<T, P>(a, s);            \
      else launch_update_tp<T, P>(a, s);                      \
      break;
    RPLU_CL_P(1) RPLU_CL_P(2) RPLU_CL_P(3) RPLU_CL_P(4)
#undef RPLU_CL_P
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_dt(int which, int32_t dtype, const CauchyLikeLaunch& a, cudaStream_t s) {
  switch (dtype) {
    case RPLU_F32: return launch_t<float>(which, a, s);
    case RPLU_F64: return launch_t<double>(which, a, s);
    case RPLU_C64: return launch_t<cf32>(which, a, s);
    case RPLU_C128: return launch_t<cf64>(which, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t cauchy_like_norms(int32_t dtype, const CauchyLikeLaunch& a, cudaStream_t s) {
  return launch_dt(0, dtype, a, s);
}

cudaError_t cauchy_like_update(int32_t dtype, const CauchyLikeLaunch& a, cudaStream_t s) {
  return launch_dt(1, dtype, a, s);
}

cudaError_t cauchy_like_finish(const CauchyLikeLaunch& a, cudaStream_t s) {
  k_cl_finish<<<1, 1024, 0, s>>>(a);
  return cudaGetLastError();
}

// Norm-kernel CTAs resident per SM for a data type and displacement rank,
// from the occupancy calculator of the current device; 0 when it cannot say.
template <typename T>
int norms_ctas_per_sm(int64_t p) {
  int nb = 0;
  cudaError_t e;
  switch (p) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cl_norms<T, 1>, kNThreads, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cl_norms<T, 2>, kNThreads, 0); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cl_norms<T, 3>, kNThreads, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cl_norms<T, 4>, kNThreads, 0); break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

// Column chunks of the norm grid (row blocks x chunks CTAs): about 8 CTAs per
// SM in all, rounded down to whole waves of resident CTAs (rounding up can
// leave a last wave of a few CTAs running alone for a whole CTA time).
int32_t cauchy_like_chunks(int64_t n, int64_t m, int32_t dtype, int64_t p, int32_t num_sms) {
  const int64_t row_blocks = std::max<int64_t>(1, (n + kNThreads * kNRows - 1) / (kNThreads * kNRows));
  const int nb = dtype == RPLU_F32 ? norms_ctas_per_sm<float>(p) : dtype == RPLU_F64 ? norms_ctas_per_sm<double>(p)
                 : dtype == RPLU_C64 ? norms_ctas_per_sm<cf32>(p) : norms_ctas_per_sm<cf64>(p);
  const int64_t target = (int64_t)num_sms * 8;
  int64_t want;
  if (nb > 0) {
    const int64_t slots = (int64_t)num_sms * nb;
    want = (target + slots - 1) / slots * slots / row_blocks;
  } else {
    want = (target + row_blocks - 1) / row_blocks;
  }
  // chunks of at least 16 columns: small problems still fill the SMs
  const int64_t max_chunks = (m + 15) / 16;
  want = std::max<int64_t>(1, std::min(want, max_chunks));
  return (int32_t)want;
}

cudaError_t cauchy_like_run(int32_t dtype, const CauchyLikeLaunch& a, cudaStream_t s, HotTimer* tm) {
  switch (dtype) {
    case RPLU_F32: return run_t<float>(a, s, tm);
    case RPLU_F64: return run_t<double>(a, s, tm);
    case RPLU_C64: return run_t<cf32>(a, s, tm);
    case RPLU_C128: return run_t<cf64>(a, s, tm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rplu
