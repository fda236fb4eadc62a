// Dense-form RPLU on the device (paper: Algorithm 1, Sec. 1; two-stage pivot
// draw of Sec. 4.1).  The residual S stays in HBM.  Per step:
//   k_dense_sample  (1 CTA)  total T = sum d, stop test, row draw by d, column
//                            draw by |S(i,:)|^2 masked on J, U(t,:) = S(i,:)
//   k_dense_update  (grid)   per row p: l_p = S(p,j)/a (FP64 division),
//                            L(p,t) = l_p, S(p,:) -= l_p U(t,:) (FMA), S(p,j) = 0,
//                            d_p = sum_q |S(p,q)|^2 -- one read and one write of S
// Rows already pivoted are exactly zero and are skipped; the current pivot row
// is not read (its update is exactly zero).
#include "common.cuh"
#include "kernels.h"
#include "sampler.cuh"

namespace rplu {
namespace {

constexpr int kUpdThreads = 256;
constexpr int kUpdMinBlocks = 4;
constexpr int kSampleThreads = 1024;

template <typename T> struct alignas(16) Vec { T v[Traits<T>::kVec]; };
static_assert(sizeof(Vec<float>) == 16 && sizeof(Vec<cf32>) == 16 && sizeof(Vec<cf64>) == 16, "16-byte vectors");

template <typename T> __device__ __forceinline__ Vec<T> as_vec(float4 r) {
  Vec<T> o;
  memcpy(&o, &r, 16);
  return o;
}
template <typename T> __device__ __forceinline__ float4 as_f4(const Vec<T>& v) {
  float4 r;
  memcpy(&r, &v, 16);
  return r;
}
// S is streamed once per step: evict-first loads and stores keep L1/L2 for the pivot row.
template <typename T> __device__ __forceinline__ Vec<T> ld_stream(const Vec<T>* p) {
  return as_vec<T>(__ldcs(reinterpret_cast<const float4*>(p)));
}
template <typename T> __device__ __forceinline__ void st_stream(Vec<T>* p, const Vec<T>& v) {
  __stcs(reinterpret_cast<float4*>(p), as_f4(v));
}
template <typename T> __device__ __forceinline__ Vec<T> ld_cached(const Vec<T>* p) {
  return as_vec<T>(__ldg(reinterpret_cast<const float4*>(p)));
}

// squared magnitude accumulated in the working precision
__device__ __forceinline__ float sq_acc(float x, float acc) { return fmaf(x, x, acc); }
__device__ __forceinline__ double sq_acc(double x, double acc) { return fma(x, x, acc); }
__device__ __forceinline__ float sq_acc(cf32 x, float acc) { return fmaf(x.im, x.im, fmaf(x.re, x.re, acc)); }
__device__ __forceinline__ double sq_acc(cf64 x, double acc) { return fma(x.im, x.im, fma(x.re, x.re, acc)); }

__device__ __forceinline__ float shfl0(float v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ double shfl0(double v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ cf32 shfl0(cf32 v) { return cf32{shfl0(v.re), shfl0(v.im)}; }
__device__ __forceinline__ cf64 shfl0(cf64 v) { return cf64{shfl0(v.re), shfl0(v.im)}; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void warp_argmax(double& v, int64_t& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double uv = __shfl_xor_sync(0xffffffffu, v, o);
    int64_t ui = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(uv, ui, v, i)) { v = uv; i = ui; }
  }
}

// Rows of this CTA: a contiguous range, so every SM gets the same share.
__device__ __forceinline__ void cta_rows(int64_t n, int64_t& r0, int64_t& r1) {
  const int64_t rpc = (n + gridDim.x - 1) / gridDim.x;
  r0 = (int64_t)blockIdx.x * rpc;
  r1 = min(n, r0 + rpc);
}

// ------------------------------------------------------------------ init
// S = A (unless in place), d_p = sum_q |A_pq|^2, non-finite check, row maxima.
template <typename T, bool kVecA, bool kComplete>
__global__ void __launch_bounds__(kUpdThreads, kUpdMinBlocks) k_dense_init(DenseLaunch a) {
  using real = typename Traits<T>::real;
  constexpr int V = Traits<T>::kVec;
  constexpr int UNR = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t r0, r1;
  cta_rows(a.n, r0, r1);
  const T* A = (const T*)a.A;
  T* S = (T*)a.S;
  const bool copy = (const void*)A != (const void*)S;
  bool bad = false;
  for (int64_t p = r0 + warp; p < r1; p += nw) {
    const T* arow = A + p * a.lda;
    T* srow = S + p * a.lds;
    double dsum = 0.0, rmax = -1.0;
    int64_t rarg = -1;
    int64_t q0 = 0;
    if (kVecA) {
      const int nvec = (int)(a.m / V);
      const Vec<T>* av = (const Vec<T>*)arow;
      Vec<T>* sv = (Vec<T>*)srow;
      for (int v0 = 0; v0 < nvec; v0 += 32 * UNR) {
        Vec<T> x[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int idx = v0 + u * 32 + lane;
          if (idx < nvec) x[u] = ld_stream(av + idx);
        }
        real acc = 0;
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int idx = v0 + u * 32 + lane;
          if (idx < nvec) {
#pragma unroll
            for (int e = 0; e < V; ++e) {
              bad |= !finite_v(x[u].v[e]);
              acc = sq_acc(x[u].v[e], acc);
              if (kComplete) {
                const double w = abs2_d(x[u].v[e]);
                if (better(w, (int64_t)idx * V + e, rmax, rarg)) { rmax = w; rarg = (int64_t)idx * V + e; }
              }
            }
            if (copy) st_stream(sv + idx, x[u]);
          }
        }
        dsum += (double)acc;
      }
      q0 = nvec * V;
    }
    for (int64_t q = q0 + lane; q < a.m; q += 32) {
      const T x = arow[q];
      bad |= !finite_v(x);
      dsum += abs2_d(x);
      if (kComplete) {
        const double w = abs2_d(x);
        if (better(w, q, rmax, rarg)) { rmax = w; rarg = q; }
      }
      if (copy) srow[q] = x;
    }
    dsum = warp_sum(dsum);
    if (kComplete) warp_argmax(rmax, rarg);
    if (lane == 0) {
      a.d[p] = dsum;
      if (kComplete) { a.rowmax[p] = rmax; a.rowarg[p] = rarg; }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) {
    atomicOr(&a.st->err, kErrNonFinite);
    a.st->done = 1;
  }
}

// ----------------------------------------------------------------- sample
// One CTA: exact fixed-point draws (sampler.cuh).  Row weights are d; column
// weights the squared entries of the drawn row with pivoted columns masked.
// While reading the row it also writes U(t,:) and its padded staging copy.
template <typename T>
__global__ void __launch_bounds__(kSampleThreads) k_dense_sample(DenseLaunch a) {
  __shared__ FxScratch sh;
  JobState* st = a.st;
  if (st->done) return;
  const int64_t t = st->t;
  const T* S = (const T*)a.S;
  const double* d = a.d;
  const uint8_t* col_used = a.col_used;
  uint64_t mb = 0;
  for (int64_t p = threadIdx.x; p < a.n; p += blockDim.x) {
    const uint64_t b = fx_bits64(d[p]);
    mb = b > mb ? b : mb;
  }
  mb = block_max_u64(mb, sh);
  const int Er = fx_scale_f64(mb, a.n);
  auto dw = [d, Er](int64_t p) -> u128 { return fx_f64(d[p], Er); };
  T* urow = (T*)a.U + t * a.m;
  T* rh = (T*)a.rhat;
  int64_t i = -1, j = -1;
  bool ok = false;
  int32_t err = 0;
  for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
    u128 Tfx;
    if (a.mode == RPLU_PIVOT_RANDOM) {
      i = fx_block_draw(dw, a.n, draw_u53(a.seed, t, 0, attempt), true, &Tfx, sh);
    } else {
      (void)fx_block_draw(dw, a.n, 0, false, &Tfx, sh);
      if (a.mode == RPLU_PIVOT_C2) {
        i = fx_block_argmax([d](int64_t p) -> uint64_t { return fx_bits64(d[p]); }, a.n, sh);
      } else if (a.mode == RPLU_PIVOT_COMPLETE) {
        const double* rm = a.rowmax;
        i = fx_block_argmax([rm](int64_t p) -> uint64_t { return fx_bits64(rm[p]); }, a.n, sh);
      } else {
        i = a.gI[t];
      }
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
    // U(t,:) = S(i,:) with pivoted columns stored as exact zeros
    const T* srow = S + i * a.lds;
    uint64_t cb = 0;
    for (int64_t q = threadIdx.x; q < a.lds; q += blockDim.x) {
      const T v = (q < a.m && !col_used[q]) ? srow[q] : zero_v<T>();
      rh[q] = v;
      if (q < a.m) urow[q] = v;
      const uint64_t b = entry_max_bits(v);
      cb = b > cb ? b : cb;
    }
    cb = block_max_u64(cb, sh);  // also orders the rhat writes before the reads below
    const int Ec = fx_entry_scale<T>(cb, a.m);
    auto cw = [rh, Ec](int64_t q) -> u128 { return fx_abs2(rh[q], Ec); };
    u128 Rfx = 1;
    if (a.mode == RPLU_PIVOT_RANDOM) {
      j = fx_block_draw(cw, a.m, draw_u53(a.seed, t, 1, attempt), true, &Rfx, sh);
    } else if (a.mode == RPLU_PIVOT_C2) {
      (void)fx_block_draw(cw, a.m, 0, false, &Rfx, sh);
      j = fx_block_argmax(cw, a.m, sh);
    } else if (a.mode == RPLU_PIVOT_COMPLETE) {
      j = a.rowarg[i];
    } else {
      j = a.gJ[t];
      if (j < 0 || j >= a.m || col_used[j]) {
        err = kErrBadGiven;
        break;
      }
    }
    if (Rfx == 0 || j < 0) {
      if (threadIdx.x == 0) a.d[i] = 0.0;
      __syncthreads();
      continue;
    }
    ok = true;
    break;
  }
  double ar = 0.0, ai = 0.0;
  if (ok) {
    to_d(S[i * a.lds + j], ar, ai);
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

// ----------------------------------------------------------------- update
template <typename T, bool kComplete>
__global__ void __launch_bounds__(kUpdThreads, kUpdMinBlocks) k_dense_update(DenseLaunch a) {
  using real = typename Traits<T>::real;
  constexpr int V = Traits<T>::kVec;
  constexpr int UNR = 4;
  const JobState* st = a.st;
  if (st->done) return;
  const int64_t t = st->cur, i = st->i, j = st->j;
  const double ar = st->a_re, ai = st->a_im;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t r0, r1;
  cta_rows(a.n, r0, r1);
  T* S = (T*)a.S;
  T* L = (T*)a.L + t * a.n;
  const Vec<T>* rv = (const Vec<T>*)a.rhat;
  const T* rh = (const T*)a.rhat;
  const int nvec = (int)(a.m / V);
  const int jv = (int)(j / V);
  const int je = (int)(j % V);
  for (int64_t p = r0 + warp; p < r1; p += nw) {
    if (a.row_used[p]) {
      if (p == i && lane == 0) {
        L[p] = one_v<T>();
        a.d[p] = 0.0;
        if (kComplete) { a.rowmax[p] = 0.0; a.rowarg[p] = -1; }
      }
      continue;
    }
    T* srow = S + p * a.lds;
    T l = zero_v<T>();
    if (lane == 0) {
      double sr, si, lr, li;
      to_d(srow[j], sr, si);
      cdiv_d(sr, si, ar, ai, lr, li);
      l = from_d<T>(lr, li);
      L[p] = l;
    }
    l = shfl0(l);
    Vec<T>* sv = (Vec<T>*)srow;
    double dsum = 0.0, rmax = -1.0;
    int64_t rarg = -1;
    for (int v0 = 0; v0 < nvec; v0 += 32 * UNR) {
      Vec<T> x[UNR], r[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int idx = v0 + u * 32 + lane;
        if (idx < nvec) {
          x[u] = ld_stream(sv + idx);
          r[u] = ld_cached(rv + idx);
        }
      }
      real acc = 0;
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int idx = v0 + u * 32 + lane;
        if (idx < nvec) {
#pragma unroll
          for (int e = 0; e < V; ++e) {
            T y = fms(x[u].v[e], l, r[u].v[e]);
            if (idx == jv && e == je) y = zero_v<T>();
            x[u].v[e] = y;
            acc = sq_acc(y, acc);
            if (kComplete) {
              const double w = abs2_d(y);
              if (better(w, (int64_t)idx * V + e, rmax, rarg)) { rmax = w; rarg = (int64_t)idx * V + e; }
            }
          }
          st_stream(sv + idx, x[u]);
        }
      }
      dsum += (double)acc;
    }
    for (int64_t q = (int64_t)nvec * V + lane; q < a.m; q += 32) {
      T y = fms(srow[q], l, rh[q]);
      if (q == j) y = zero_v<T>();
      srow[q] = y;
      dsum += abs2_d(y);
      if (kComplete) {
        const double w = abs2_d(y);
        if (better(w, q, rmax, rarg)) { rmax = w; rarg = q; }
      }
    }
    dsum = warp_sum(dsum);
    if (kComplete) warp_argmax(rmax, rarg);
    if (lane == 0) {
      a.d[p] = dsum;
      if (kComplete) { a.rowmax[p] = rmax; a.rowarg[p] = rarg; }
    }
  }
}

// ----------------------------------------------------------------- finish
__global__ void __launch_bounds__(kSampleThreads) k_dense_finish(const double* d, int64_t n, double* T_hist,
                                                               JobState* st) {
  __shared__ FxScratch sh;
  const double T = fx_total_f64(d, n, sh);
  if (threadIdx.x == 0) {
    if (!st->done) {
      st->done = 1;
      st->k_done = st->t;
    }
    T_hist[st->k_done] = T;
    if (st->k_done == 0 && st->t == 0) st->T0 = T;
  }
}

template <typename T>
cudaError_t dense_run_t(const DenseLaunch& a, cudaStream_t s, HotTimer* tm) {
  constexpr int V = Traits<T>::kVec;
  const bool complete = a.mode == RPLU_PIVOT_COMPLETE;
  const int64_t warps = kUpdThreads / 32;
  int64_t grid = (a.n + warps - 1) / warps;
  const int64_t cap = (int64_t)a.num_sms * kUpdMinBlocks;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  const bool vecA = ((uintptr_t)a.A % 16 == 0) && ((a.lda * (int64_t)sizeof(T)) % 16 == 0) && a.m >= V;
  if (a.n > 0 && a.m > 0) {
    if (vecA) {
      if (complete) k_dense_init<T, true, true><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
      else k_dense_init<T, true, false><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
    } else {
      if (complete) k_dense_init<T, false, true><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
      else k_dense_init<T, false, false><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
    }
    tm->all_launches += 1;
  }
  for (int64_t t = 0; t < a.k; ++t) {
    k_dense_sample<T><<<1, kSampleThreads, 0, s>>>(a);
    tm->begin();
    if (complete) k_dense_update<T, true><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
    else k_dense_update<T, false><<<(unsigned)grid, kUpdThreads, 0, s>>>(a);
    tm->end();
    tm->all_launches += 2;
  }
  k_dense_finish<<<1, kSampleThreads, 0, s>>>(a.d, a.n, a.T_hist, a.st);
  tm->all_launches += 1;
  return cudaGetLastError();
}

}  // namespace

cudaError_t dense_run(int32_t dtype, const DenseLaunch& a, cudaStream_t s, HotTimer* tm) {
  switch (dtype) {
    case RPLU_F32: return dense_run_t<float>(a, s, tm);
    case RPLU_F64: return dense_run_t<double>(a, s, tm);
    case RPLU_C64: return dense_run_t<cf32>(a, s, tm);
    case RPLU_C128: return dense_run_t<cf64>(a, s, tm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rplu
