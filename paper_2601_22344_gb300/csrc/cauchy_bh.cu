// Algorithm 3 (Sec. 5.1) with its row draw by rejection sampling against the
// row-norm upper bounds of App. C.  The quadtrees and interaction lists
// (Algorithm C.1) are built once on the host (bh_plan.h); every step then runs
//
//   k_bh_gram     (grid)   Gram matrices H_s = sum_{j in s} B(:,j) B(:,j)^* of
//                          every source node, bottom-up: one warp per source
//                          leaf sums its points, and the warp that completes a
//                          node's last child sums the children (arrival counters)
//   k_bh_bounds   (grid)   one CTA per target leaf l (Algorithm C.2):
//                          M_l = sum_{(s,alpha) in A_l} alpha H_s, then for each
//                          point i of l, u_i = G(i,:) M_l G(i,:)^* plus the exact
//                          terms |G(i,:) B(:,j)|^2 / |x_i - y_j|^2 of the source
//                          leaves in E_l
//   k_bh_sample   (1 CTA)  sum of u and the stop test; proposals i ~ u, the exact
//                          row r = S(i,:) and rho = ||r||^2, acceptance when
//                          V u_i < rho; the column j ~ |r_j|^2 of the accepted row
//   [exact-norm pass and k_bh_fallback, only for a step whose 64 proposals were
//    all rejected: the exact-norm draw of that step]
//   k_cl_update   (grid)   L column and generator updates (cauchy_like.cu)
//
// The order of the terms differs from a literal reading of Algorithm C.2 (the
// aggregated Gram matrices of a leaf are combined before the quadratic form),
// which changes the bounds only by rounding.  The quadratic forms and Gram
// matrices are FP64 for every data type; the exact near-field terms use the
// working precision with FP64 sums across source chunks.
#include "cauchy_like.cuh"
#include "common.cuh"
#include "kernels.h"
#include "sampler.cuh"

namespace rplu {
namespace {

constexpr int kGWarps = 4;        // Gram kernel: warps per CTA, one source leaf each
constexpr int kBThreads = 128;    // bounds kernel: one target leaf per CTA
constexpr int kBWarps = kBThreads / 32;
constexpr int kBStage = 256;      // source points staged in shared memory at a time
constexpr int kSThreads = 1024;   // single-CTA draw kernels
// Stream of the acceptance uniforms and of the exact-norm fallback draw
// (the proposals use the plain seed).
constexpr uint64_t kAccStream = 0xA0761D6478BD642Full;

__device__ __forceinline__ double sel_lane(const double* v, int n, int lane) {
  double r = 0.0;
#pragma unroll
  for (int e = 0; e < 32; ++e)
    if (e < n && e == lane) r = v[e];
  return r;
}

// ------------------------------------------------------------------ Gram
template <typename T, int P>
__global__ void __launch_bounds__(kGWarps * 32) k_bh_gram(CauchyLikeLaunch a, BhLaunch b) {
  constexpr int E2 = 2 * P * P;  // doubles per Gram matrix
  if (a.st->done) return;
  const int lane = threadIdx.x & 31;
  const int leaf = blockIdx.x * kGWarps + (threadIdx.x >> 5);
  if (leaf >= b.n_sleaf) return;
  const T* Bm = (const T*)a.B;
  int node = b.sleaf[leaf];
  const int2 rg = b.snode[node];
  double h[E2];
#pragma unroll
  for (int e = 0; e < E2; ++e) h[e] = 0.0;
  for (int q = rg.x + lane; q < rg.y; q += 32) {
    const int64_t j = b.sperm[q];
    double br[P], bi[P];
#pragma unroll
    for (int l = 0; l < P; ++l) to_d(Bm[(int64_t)l * a.m + j], br[l], bi[l]);
    // H(r, c) += B_r conj(B_c)
#pragma unroll
    for (int r = 0; r < P; ++r)
#pragma unroll
      for (int c = 0; c < P; ++c) {
        h[2 * (r * P + c)] = fma(br[r], br[c], fma(bi[r], bi[c], h[2 * (r * P + c)]));
        h[2 * (r * P + c) + 1] = fma(bi[r], br[c], fma(-br[r], bi[c], h[2 * (r * P + c) + 1]));
      }
  }
#pragma unroll
  for (int e = 0; e < E2; ++e)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h[e] += __shfl_xor_sync(0xffffffffu, h[e], o);
  const double mine = sel_lane(h, E2, lane);
  if (lane < E2) b.H[(int64_t)node * E2 + lane] = mine;
  // climb: the warp whose arrival completes a parent sums its children
  __threadfence();
  int parent = b.sparent[node];
  while (parent >= 0) {
    int last = 0;
    if (lane == 0) last = atomicAdd(&b.cnt[parent], 1) == b.snchild[parent] - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) break;
    __threadfence();
    if (lane == 0) b.cnt[parent] = 0;  // every child has arrived: ready for the next step
    const int4 ch = b.schild[parent];
    if (lane < E2) {
      double acc = 0.0;
      if (ch.x >= 0) acc += __ldcg(&b.H[(int64_t)ch.x * E2 + lane]);
      if (ch.y >= 0) acc += __ldcg(&b.H[(int64_t)ch.y * E2 + lane]);
      if (ch.z >= 0) acc += __ldcg(&b.H[(int64_t)ch.z * E2 + lane]);
      if (ch.w >= 0) acc += __ldcg(&b.H[(int64_t)ch.w * E2 + lane]);
      b.H[(int64_t)parent * E2 + lane] = acc;
    }
    __threadfence();
    node = parent;
    parent = b.sparent[node];
  }
}

// ---------------------------------------------------------------- bounds
// Near-field term |sum_l g_l b_l|^2 / |x - y|^2 in the working precision.
template <typename T, int P>
__device__ __forceinline__ typename Traits<T>::real near_term(const T (&g)[P], const T* bq, int stride, T x, T y) {
  using real = typename Traits<T>::real;
  T sv = mul_v(g[0], bq[0]);
#pragma unroll
  for (int l = 1; l < P; ++l) sv = add_v(sv, mul_v(g[l], bq[(int64_t)l * stride]));
  const real zr = re_of(x) - re_of(y), zi = im_of(x) - im_of(y);
  const real sr = re_of(sv), si = im_of(sv);
  return (sr * sr + si * si) * rcp_fast(zr * zr + zi * zi);
}

template <typename T, int P>
__global__ void __launch_bounds__(kBThreads) k_bh_bounds(CauchyLikeLaunch a, BhLaunch b) {
  using real = typename Traits<T>::real;
  constexpr int E2 = 2 * P * P;
  __shared__ double Ms[E2];
  __shared__ T sy[kBStage];
  __shared__ T sb[P * kBStage];
  __shared__ double part[kBWarps][32];
  if (a.st->done) return;
  const int lf = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  const T* G = (const T*)a.G;
  const T* Bm = (const T*)a.B;
  if (threadIdx.x < E2) {
    double acc = 0.0;
    for (int e = b.a_off[lf]; e < b.a_off[lf + 1]; ++e)
      acc = fma(b.a_alpha[e], b.H[(int64_t)b.a_node[e] * E2 + threadIdx.x], acc);
    Ms[threadIdx.x] = acc;
  }
  const int2 tl = b.tleaf[lf];
  const int e0 = b.e_off[lf], e1 = b.e_off[lf + 1];
  for (int pbase = tl.x; pbase < tl.y; pbase += 32) {
    const int pos = pbase + lane;
    const bool live = pos < tl.y;
    const int64_t i = b.tperm[live ? pos : tl.x];
    const T xi = x[i];
    T g[P];
#pragma unroll
    for (int l = 0; l < P; ++l) g[l] = G[i * P + l];
    double accn = 0.0;
    // stage the points of the exact source leaves, kBStage at a time
    int ce = e0;
    int cq = ce < e1 ? b.snode[b.e_node[ce]].x : 0;
    while (ce < e1) {
      __syncthreads();
      int filled = 0;
      while (ce < e1 && filled < kBStage) {
        const int2 r = b.snode[b.e_node[ce]];
        const int take = min(r.y - cq, kBStage - filled);
        for (int q = threadIdx.x; q < take; q += kBThreads) {
          const int64_t j = b.sperm[cq + q];
          sy[filled + q] = y[j];
#pragma unroll
          for (int l = 0; l < P; ++l) sb[l * kBStage + filled + q] = Bm[(int64_t)l * a.m + j];
        }
        filled += take;
        cq += take;
        if (cq >= r.y) {
          ++ce;
          if (ce < e1) cq = b.snode[b.e_node[ce]].x;
        }
      }
      __syncthreads();
      real acc = 0;
      for (int q = warp; q < filled; q += kBWarps) acc += near_term<T, P>(g, &sb[q], kBStage, xi, sy[q]);
      accn += (double)acc;
    }
    part[warp][lane] = accn;
    __syncthreads();
    if (warp == 0 && live) {
      double near = part[0][lane];
#pragma unroll
      for (int w = 1; w < kBWarps; ++w) near += part[w][lane];
      // G(i,:) M G(i,:)^*: real part of sum_{r,c} g_r M_rc conj(g_c)
      double far = 0.0;
#pragma unroll
      for (int r = 0; r < P; ++r) {
        double gr, gi;
        to_d(g[r], gr, gi);
#pragma unroll
        for (int c = 0; c < P; ++c) {
          double cr, ci;
          to_d(g[c], cr, ci);
          const double mr = Ms[2 * (r * P + c)], mi = Ms[2 * (r * P + c) + 1];
          // Re[(gr + i gi)(mr + i mi)(cr - i ci)]
          const double pr = gr * mr - gi * mi, pi = gr * mi + gi * mr;
          far += pr * cr + pi * ci;
        }
      }
      b.u[i] = far + near;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ draw
// r = S(i,:) from the generators with the pivoted columns masked; returns
// the fixed-point scale of |r_q|^2 (the block barrier inside also orders the
// writes of r before any read).
template <typename T, int P>
__device__ int gen_row(const CauchyLikeLaunch& a, int64_t i, FxScratch& sh) {
  const T* x = (const T*)a.x;
  const T* y = (const T*)a.y;
  const T* G = (const T*)a.G;
  const T* Bm = (const T*)a.B;
  T* r = (T*)a.r;
  T gi[P];
#pragma unroll
  for (int l = 0; l < P; ++l) gi[l] = G[i * P + l];
  const T xi = x[i];
  uint64_t cb = 0;
  for (int64_t q = threadIdx.x; q < a.m; q += blockDim.x) {
    T bq[P];
#pragma unroll
    for (int l = 0; l < P; ++l) bq[l] = Bm[(int64_t)l * a.m + q];
    const T v = a.col_used[q] ? zero_v<T>() : entry_gen<T, P>(gi, bq, xi, y[q]);
    r[q] = v;
    const uint64_t bits = entry_max_bits(v);
    cb = bits > cb ? bits : cb;
  }
  cb = block_max_u64(cb, sh);
  return fx_entry_scale<T>(cb, a.m);
}

// Records the pivot (i, j) of step t: U(t,:) = r, saved G(i,:) and B(:,j),
// masks and state for the update kernel.  Returns false (and ends the
// factorization) on a zero pivot value.
template <typename T, int P>
__device__ bool commit_pivot(const CauchyLikeLaunch& a, const BhLaunch& b, int64_t t, int64_t i, int64_t j,
                             int32_t attempts) {
  JobState* st = a.st;
  const T* r = (const T*)a.r;
  double ar, ai;
  to_d(r[j], ar, ai);
  if (ar == 0.0 && ai == 0.0) {
    if (threadIdx.x == 0) {
      st->done = 1;
      st->k_done = t;
      atomicOr(&st->err, kErrZeroPivot);
    }
    return false;
  }
  T* urow = (T*)a.U + t * a.m;
  for (int64_t q = threadIdx.x; q < a.m; q += blockDim.x) urow[q] = r[q];
  const T* G = (const T*)a.G;
  const T* Bm = (const T*)a.B;
  if (threadIdx.x < P) {
    ((T*)a.gi)[threadIdx.x] = G[i * P + threadIdx.x];
    ((T*)a.bj)[threadIdx.x] = Bm[(int64_t)threadIdx.x * a.m + j];
  }
  if (threadIdx.x == 0) {
    a.col_used[j] = 1;
    a.row_used[i] = 1;
    a.I[t] = i;
    a.J[t] = j;
    if (b.attempts) b.attempts[t] = attempts;
    st->i = i;
    st->j = j;
    st->a_re = ar;
    st->a_im = ai;
    st->cur = t;
    st->t = t + 1;
    st->fallback = 0;
  }
  return true;
}

__device__ __forceinline__ void stop_at(JobState* st, int64_t t) {
  if (threadIdx.x == 0) {
    st->done = 1;
    st->k_done = t;
  }
}

template <typename T, int P>
__global__ void __launch_bounds__(kSThreads) k_bh_sample(CauchyLikeLaunch a, BhLaunch b) {
  __shared__ FxScratch shu;
  __shared__ FxScratch sh;
  JobState* st = a.st;
  if (st->done) return;
  const int64_t t = st->t;
  const double* u = b.u;
  uint64_t mb = max_bits_f64(u, a.n);
  mb = block_max_u64(mb, shu);
  const int Eu = fx_scale_f64(mb, a.n);
  auto uw = [u, Eu](int64_t p) -> u128 { return fx_f64(u[p], Eu); };
  fx_block_totals(uw, a.n, shu);
  u128 Ufx;
  (void)fx_block_pick(uw, a.n, 0, 0, (u128)0, &Ufx, shu);
  const double Us = fx_to_double(Ufx, Eu);
  if (threadIdx.x == 0) a.T_hist[t] = Us;
  if (!(Us > 0.0) || (a.tol > 0.0 && Us <= a.tol * a.tol * st->T0)) {
    stop_at(st, t);
    return;
  }
  const T* rr = (const T*)a.r;
  for (int att = 0; att < kMaxAttempts; ++att) {
    const int64_t i = fx_block_pick(uw, a.n, 1, draw_u53(a.seed, t, 0, att), (u128)0, &Ufx, shu);
    if (i < 0) break;
    const int Ec = gen_row<T, P>(a, i, sh);
    auto cw = [rr, Ec](int64_t q) -> u128 { return fx_abs2(rr[q], Ec); };
    fx_block_totals(cw, a.m, sh);
    u128 Rfx;
    (void)fx_block_pick(cw, a.m, 0, 0, (u128)0, &Rfx, sh);
    const double rho = fx_to_double(Rfx, Ec);
    const double V = (double)draw_u53(a.seed ^ kAccStream, t, 0, att) * 0x1p-53;
    if (!(rho > 0.0) || !(V * u[i] < rho)) continue;
    const int64_t j = fx_block_pick(cw, a.m, 1, draw_u53(a.seed, t, 1, att), (u128)0, &Rfx, sh);
    if (j < 0) break;
    (void)commit_pivot<T, P>(a, b, t, i, j, att + 1);
    return;
  }
  if (threadIdx.x == 0) st->fallback = 1;
}

// The exact-norm draw of a step whose proposals were all rejected; the exact
// squared row norms d of the residual come from the (gated) norm pass before.
template <typename T, int P>
__global__ void __launch_bounds__(kSThreads) k_bh_fallback(CauchyLikeLaunch a, BhLaunch b) {
  __shared__ FxScratch sh;
  JobState* st = a.st;
  if (st->done || !st->fallback) return;
  const int64_t t = st->t;
  const double* d = a.d;
  uint64_t mb = max_bits_f64(d, a.n);
  mb = block_max_u64(mb, sh);
  const int Er = fx_scale_f64(mb, a.n);
  u128 Tfx;
  const int64_t i = fx_block_draw([d, Er](int64_t p) -> u128 { return fx_f64(d[p], Er); }, a.n,
                                  draw_u53(a.seed ^ kAccStream, t, 1, 0), true, &Tfx, sh);
  if (Tfx == 0 || i < 0) {
    stop_at(st, t);
    return;
  }
  const int Ec = gen_row<T, P>(a, i, sh);
  const T* rr = (const T*)a.r;
  u128 Rfx;
  const int64_t j = fx_block_draw([rr, Ec](int64_t q) -> u128 { return fx_abs2(rr[q], Ec); }, a.m,
                                  draw_u53(a.seed ^ kAccStream, t, 1, 1), true, &Rfx, sh);
  if (Rfx == 0 || j < 0) {
    stop_at(st, t);
    return;
  }
  (void)commit_pivot<T, P>(a, b, t, i, j, kMaxAttempts + 1);
}

// T0 = exact ||A||_F^2 from the initial exact norms.
__global__ void k_bh_t0(CauchyLikeLaunch a) {
  __shared__ FxScratch sh;
  const double T_ = fx_total_f64(a.d, a.n, sh);
  if (threadIdx.x == 0) a.st->T0 = T_;
}

template <typename T, int P>
void launch_bounds_tp(const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm) {
  const unsigned gg = (unsigned)((b.n_sleaf + kGWarps - 1) / kGWarps);
  k_bh_gram<T, P><<<std::max(gg, 1u), kGWarps * 32, 0, s>>>(a, b);
  if (tm) tm->begin();
  k_bh_bounds<T, P><<<(unsigned)std::max(b.n_tleaf, 1), kBThreads, 0, s>>>(a, b);
  if (tm) {
    tm->end();
    tm->all_launches += 2;
  }
}

template <typename T, int P>
cudaError_t run_tp(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm) {
  CauchyLikeLaunch forced = a, gated = a;
  forced.gate = kGateForced;
  gated.gate = kGateFallback;
  cudaError_t e = cauchy_like_norms(dtype, forced, s);
  if (e != cudaSuccess) return e;
  k_bh_t0<<<1, 1024, 0, s>>>(a);
  tm->all_launches += 3;
  for (int64_t t = 0; t < a.k; ++t) {
    launch_bounds_tp<T, P>(a, b, s, tm);
    k_bh_sample<T, P><<<1, kSThreads, 0, s>>>(a, b);
    e = cauchy_like_norms(dtype, gated, s);
    if (e != cudaSuccess) return e;
    k_bh_fallback<T, P><<<1, kSThreads, 0, s>>>(a, b);
    e = cauchy_like_update(dtype, a, s);
    if (e != cudaSuccess) return e;
    tm->all_launches += 5;
  }
  e = cauchy_like_norms(dtype, forced, s);
  if (e != cudaSuccess) return e;
  e = cauchy_like_finish(a, s);
  tm->all_launches += 3;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_t(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm,
                  bool bounds_only) {
  switch (a.p) {
#define RPLU_BH_P(P)                                              \
    case P:                                                       \
      if (bounds_only) {                                          \
        launch_bounds_tp<T, P>(a, b, s, nullptr);                 \
        return cudaGetLastError();                                \
      }                                                           \
      return run_tp<T, P>(dtype, a, b, s, tm);
    RPLU_BH_P(1) RPLU_BH_P(2) RPLU_BH_P(3) RPLU_BH_P(4)
#undef RPLU_BH_P
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t run_dt(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm,
                   bool bounds_only) {
  switch (dtype) {
    case RPLU_F32: return run_t<float>(dtype, a, b, s, tm, bounds_only);
    case RPLU_F64: return run_t<double>(dtype, a, b, s, tm, bounds_only);
    case RPLU_C64: return run_t<cf32>(dtype, a, b, s, tm, bounds_only);
    case RPLU_C128: return run_t<cf64>(dtype, a, b, s, tm, bounds_only);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t cauchy_like_bh_run(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s,
                               HotTimer* tm) {
  return run_dt(dtype, a, b, s, tm, false);
}

cudaError_t cauchy_like_bh_bounds(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s) {
  return run_dt(dtype, a, b, s, nullptr, true);
}

}  // namespace rplu
