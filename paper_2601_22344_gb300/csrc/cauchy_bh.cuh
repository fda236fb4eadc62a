// Algorithm 3 (Sec. 5.1) with its row draw by rejection sampling against the
// row-norm upper bounds of App. C.  The quadtrees and interaction lists
// (Algorithm C.1) are built once on the host (bh_plan.h); every step then runs
//
//   k_bh_gram_leaf (grid)  Gram matrices H_s = sum_{j in s} B(:,j) B(:,j)^* of
//                          the source leaves, one warp per leaf
//   k_bh_gram_nodes (grid) H_s of every internal source node as the sum of
//                          the leaf Grams under it, one warp per node
//   k_bh_bounds   (grid)   one CTA per target leaf l (Algorithm C.2):
//                          M_l = sum_{(s,alpha) in A_l} alpha H_s, then for each
//                          point i of l, u_i = G(i,:) M_l G(i,:)^* plus the exact
//                          terms |G(i,:) B(:,j)|^2 / |x_i - y_j|^2 of the source
//                          leaves in E_l
//   k_bh_sample   (cluster of 8 CTAs) sum of u and the stop test; proposals
//                          i ~ u, the exact row r = S(i,:) and rho = ||r||^2,
//                          acceptance when V u_i < rho; the column j ~ |r_j|^2
//                          of the accepted row
//   [exact-norm pass and k_bh_fallback, only for a step whose 64 proposals were
//    all rejected: the exact-norm draw of that step]
//   k_cl_update   (grid)   L column and generator updates (cauchy_like.cu)
//
// The order of the terms differs from a literal reading of Algorithm C.2 (the
// aggregated Gram matrices of a leaf are combined before the quadratic form),
// which changes the bounds only by rounding.  The quadratic forms and Gram
// matrices are FP64 for every data type; the exact near-field terms use the
// working precision with FP64 sums across source chunks.
//
// Shared by the per-dtype translation units cauchy_bh_{f32,f64,c64,c128}.cu,
// which instantiate these templates for one data type each (compiled in
// parallel), and the dispatcher cauchy_bh.cu.
#pragma once

#include <cstring>

#include "cauchy_like.cuh"
#include "common.cuh"
#include "cluster.cuh"
#include "kernels.h"
#include "rcp.cuh"
#include "sampler.cuh"

namespace rplu {
namespace {

constexpr int kGWarps = 4;        // Gram kernel: warps per CTA, one source leaf each
constexpr int kBThreads = 256;    // bounds kernel: one target leaf (slice) per CTA
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
// Leaf pass: one warp per source leaf sums B(:,j) B(:,j)^* over its points
// (FP64, lanes strided, then a fixed xor tree).
template <typename T, int P>
__global__ void __launch_bounds__(kGWarps * 32) k_bh_gram_leaf(CauchyLikeLaunch a, BhLaunch b) {
  constexpr int E2 = 2 * P * P;  // doubles per Gram matrix
  if (a.st->done) return;
  const int lane = threadIdx.x & 31;
  const int leaf = blockIdx.x * kGWarps + (threadIdx.x >> 5);
  if (leaf >= b.n_sleaf) return;
  const T* Bm = (const T*)a.B;
  const int node = b.sleaf[leaf];
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
}

// Node pass: one warp per internal source node sums the Gram matrices of the
// leaves under it (a contiguous run of the leaf list, which is in tree
// order), lanes strided over the leaves, then a fixed xor tree.  The bottom-up
// traversal of Algorithm C.2 in one level: every node reads only leaf sums.
template <int P>
__global__ void __launch_bounds__(kGWarps * 32) k_bh_gram_nodes(CauchyLikeLaunch a, BhLaunch b) {
  constexpr int E2 = 2 * P * P;
  if (a.st->done) return;
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * kGWarps + (threadIdx.x >> 5);
  if (w >= b.n_sinner) return;
  const int node = b.sinner[w];
  const int2 lr = b.sleafrange[node];
  double h[E2];
#pragma unroll
  for (int e = 0; e < E2; ++e) h[e] = 0.0;
  for (int l = lr.x + lane; l < lr.y; l += 32) {
    const double* hl = b.H + (int64_t)b.sleaf[l] * E2;
#pragma unroll
    for (int e = 0; e < E2; ++e) h[e] += hl[e];
  }
#pragma unroll
  for (int e = 0; e < E2; ++e)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h[e] += __shfl_xor_sync(0xffffffffu, h[e], o);
  const double mine = sel_lane(h, E2, lane);
  if (lane < E2) b.H[(int64_t)node * E2 + lane] = mine;
}

// ---------------------------------------------------------------- bounds
// Near-field term |sum_l g_l b_l|^2 / |x - y|^2 in the working precision.
// FP32 data: the hardware reciprocal; FP64 data: sums of products as FMA
// chains and the two-step Newton reciprocal (rcp.cuh), fewer FP64
// instructions than complex multiply-adds and an IEEE division.
template <int P, typename T>
__device__ __forceinline__ typename Traits<T>::real near_term(const T (&g)[P], const T* bq, int stride, T x, T y) {
  using real = typename Traits<T>::real;
  T sv = mul_v(g[0], bq[0]);
#pragma unroll
  for (int l = 1; l < P; ++l) sv = add_v(sv, mul_v(g[l], bq[(int64_t)l * stride]));
  const real zr = re_of(x) - re_of(y), zi = im_of(x) - im_of(y);
  const real sr = re_of(sv), si = im_of(sv);
  return (sr * sr + si * si) * rcp_fast(zr * zr + zi * zi);
}
template <int P>
__device__ __forceinline__ double near_term(const double (&g)[P], const double* bq, int stride, double x, double y) {
  double sv = g[0] * bq[0];
#pragma unroll
  for (int l = 1; l < P; ++l) sv = fma(g[l], bq[(int64_t)l * stride], sv);
  const double z = x - y;
  return (sv * sv) * rcp_nr64(z * z);
}
template <int P>
__device__ __forceinline__ double near_term(const cf64 (&g)[P], const cf64* bq, int stride, cf64 x, cf64 y) {
  double sr = g[0].re * bq[0].re, si = g[0].re * bq[0].im;
  sr = fma(-g[0].im, bq[0].im, sr);
  si = fma(g[0].im, bq[0].re, si);
#pragma unroll
  for (int l = 1; l < P; ++l) {
    const cf64 b = bq[(int64_t)l * stride];
    sr = fma(g[l].re, b.re, sr);
    sr = fma(-g[l].im, b.im, sr);
    si = fma(g[l].re, b.im, si);
    si = fma(g[l].im, b.re, si);
  }
  const double zr = x.re - y.re, zi = x.im - y.im;
  return fma(sr, sr, si * si) * rcp_nr64(fma(zr, zr, zi * zi));
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
  const int slice = blockIdx.y;
  if (threadIdx.x < E2) {
    double acc = 0.0;
    if (slice == 0)
      for (int e = b.a_off[lf]; e < b.a_off[lf + 1]; ++e)
        acc = fma(b.a_alpha[e], b.H[(int64_t)b.a_node[e] * E2 + threadIdx.x], acc);
    Ms[threadIdx.x] = acc;
  }
  const int2 tl = b.tleaf[lf];
  // this slice's share of the exact source leaves
  const int ea = b.e_off[lf], eb = b.e_off[lf + 1];
  const int e0 = ea + (int)((int64_t)(eb - ea) * slice / gridDim.y);
  const int e1 = ea + (int)((int64_t)(eb - ea) * (slice + 1) / gridDim.y);
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
      for (int q = warp; q < filled; q += kBWarps) acc += near_term<P>(g, &sb[q], kBStage, xi, sy[q]);
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
      b.u[(int64_t)slice * a.n + i] = far + near;
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

// The bound of row p: the sum of the slices' partial bounds, in slice order.
__device__ __forceinline__ double u_at(const double* u, int ns, int64_t n, int64_t p) {
  double v = u[p];
  for (int s = 1; s < ns; ++s) v += u[(int64_t)s * n + p];
  return v;
}

// The draw of step t on a cluster of kCl CTAs: CTA c owns rows
// [c RS, (c+1) RS) of u and columns [c CS, (c+1) CS) of the proposed row.
// Per proposal: cluster-wide exact row draw over u, the row r = S(i,:) on
// each CTA's columns, the cluster-wide exact column draw over |r_q|^2 (whose
// total is rho), and the acceptance V u_i < rho, taken alike in every CTA.
// The column uniform does not depend on the acceptance, so drawing the column
// before deciding gives the column of the accepted proposal.
template <typename T, int P>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClThreads) k_bh_sample(CauchyLikeLaunch a, BhLaunch b) {
  __shared__ FxScratch sh;
  __shared__ ClShared x;
  JobState* st = a.st;
  const uint32_t rank = cl_rank();
  const bool lead = rank == 0 && threadIdx.x == 0;
  if (st->done) {  // same value in every CTA: nothing writes it before the final barrier
    if (lead && b.use_graph) cudaGraphSetConditional(b.h_fb, 0u);
    return;
  }
  const int64_t t = st->t;
  const int64_t n = a.n, m = a.m;
  const double* u = b.u;
  const int ns = b.nslice;
  const int64_t RS = (n + kCl - 1) / kCl;
  const int64_t rlo = min(n, (int64_t)rank * RS), rlen = min(n, rlo + RS) - rlo;
  const int64_t CS = (m + kCl - 1) / kCl;
  const int64_t qlo = min(m, (int64_t)rank * CS), qlen = min(m, qlo + CS) - qlo;
  const T* x_ = (const T*)a.x;
  const T* y = (const T*)a.y;
  const T* G = (const T*)a.G;
  const T* Bm = (const T*)a.B;
  T* r = (T*)a.r;
  int ex = 0;
  uint64_t mb = 0;
  for (int64_t p = rlo + threadIdx.x; p < rlo + rlen; p += kClThreads) {
    const uint64_t bits = fx_bits64(u_at(u, ns, n, p));
    mb = bits > mb ? bits : mb;
  }
  const uint64_t gmb = cl_max(mb, x, sh, rank, ex);
  const int Eu = fx_scale_f64(gmb, n);
  auto uw = [u, ns, n, Eu](int64_t p) -> u128 { return fx_f64(u_at(u, ns, n, p), Eu); };
  // the stopping test: sum(u) <= tol^2 T0, or (max rule) max(u) <= tol^2 max(u at step 0)
  const double umax = __longlong_as_double((long long)gmb);
  const double umax0 = t == 0 ? umax : *b.umax0;
  if (t == 0 && lead) *b.umax0 = umax;
  auto stop_test = [&](double Us) {
    if (!(Us > 0.0)) return true;
    if (!(a.tol > 0.0)) return false;
    return b.stop_max ? umax <= a.tol * a.tol * umax0 : Us <= a.tol * a.tol * st->T0;
  };
  int64_t i = -1, j = -1;
  int outcome = 0;  // 0: every proposal rejected, 1: accepted, 2: stop
  int32_t att = 0;
  const T* rr = r;
  if (a.mode == RPLU_PIVOT_C2) {
    // approximate C2PLU (Sec. 5.1): the row of the largest bound, then the
    // largest entry of its row; a row with no weight left is set aside
    __shared__ int64_t excl[kMaxAttempts];
    int nex = 0;
    const double Us = fx_to_double(cl_total(uw, rlo, rlen, x, sh, rank, ex), Eu);
    if (lead) a.T_hist[t] = Us;
    outcome = stop_test(Us) ? 2 : 0;
    for (; outcome == 0 && att < kMaxAttempts; ++att) {
      auto ukey = [u, ns, n, &nex](int64_t p) -> uint64_t {
        for (int e = 0; e < nex; ++e)
          if (excl[e] == p) return 0ull;
        return fx_bits64(u_at(u, ns, n, p));
      };
      uint64_t key;
      i = cl_argmax(ukey, rlo, rlen, x, sh, rank, ex, &key);
      if (i < 0) break;
      T gi[P];
#pragma unroll
      for (int l = 0; l < P; ++l) gi[l] = G[i * P + l];
      const T xi = x_[i];
      for (int64_t q = qlo + threadIdx.x; q < qlo + qlen; q += kClThreads) {
        T bq[P];
#pragma unroll
        for (int l = 0; l < P; ++l) bq[l] = Bm[(int64_t)l * m + q];
        r[q] = a.col_used[q] ? zero_v<T>() : entry_gen<T, P>(gi, bq, xi, y[q]);
      }
      __syncthreads();
      auto rkey = [rr](int64_t q) -> uint64_t { return fx_bits64(abs2_d(rr[q])); };
      j = cl_argmax(rkey, qlo, qlen, x, sh, rank, ex, &key);
      if (j < 0) {
        if (threadIdx.x == 0 && nex < kMaxAttempts) excl[nex] = i;
        ++nex;
        __syncthreads();
        continue;
      }
      outcome = 1;
      break;
    }
    if (outcome == 0) outcome = 2;  // no row with weight left
  }
  for (; a.mode != RPLU_PIVOT_C2 && att < kMaxAttempts; ++att) {
    u128 Ufx;
    i = cl_draw(uw, rlo, rlen, draw_u53(a.seed, t, 0, att), &Ufx, x, sh, rank, ex);
    if (att == 0) {
      const double Us = fx_to_double(Ufx, Eu);
      if (lead) a.T_hist[t] = Us;
      if (stop_test(Us)) {
        outcome = 2;
        break;
      }
    }
    if (i < 0) break;
    // r = S(i,:) on this CTA's columns, pivoted columns masked
    T gi[P];
#pragma unroll
    for (int l = 0; l < P; ++l) gi[l] = G[i * P + l];
    const T xi = x_[i];
    uint64_t cb = 0;
    for (int64_t q = qlo + threadIdx.x; q < qlo + qlen; q += kClThreads) {
      T bq[P];
#pragma unroll
      for (int l = 0; l < P; ++l) bq[l] = Bm[(int64_t)l * m + q];
      const T v = a.col_used[q] ? zero_v<T>() : entry_gen<T, P>(gi, bq, xi, y[q]);
      r[q] = v;
      const uint64_t bits = entry_max_bits(v);
      cb = bits > cb ? bits : cb;
    }
    const int Ec = fx_entry_scale<T>(cl_max(cb, x, sh, rank, ex), m);  // its barrier orders the writes of r
    auto cw = [rr, Ec](int64_t q) -> u128 { return fx_abs2(rr[q], Ec); };
    u128 Rfx;
    j = cl_draw(cw, qlo, qlen, draw_u53(a.seed, t, 1, att), &Rfx, x, sh, rank, ex);
    const double rho = fx_to_double(Rfx, Ec);
    const double V = (double)draw_u53(a.seed ^ kAccStream, t, 0, att) * 0x1p-53;
    if (rho > 0.0 && V * u_at(u, ns, n, i) < rho && j >= 0) {
      outcome = 1;
      break;
    }
  }
  if (outcome == 1) {
    // U(t,:) = r: every CTA copies its own columns
    T* urow = (T*)a.U + t * m;
    for (int64_t q = qlo + threadIdx.x; q < qlo + qlen; q += kClThreads) urow[q] = r[q];
  }
  cl_sync();  // r(j), written by the CTA that owns column j, is visible to CTA 0
  if (rank != 0) return;
  if (outcome == 1) {
    double ar, ai;
    to_d(ld_l2(r + j), ar, ai);
    if (ar == 0.0 && ai == 0.0) {
      if (threadIdx.x == 0) {
        st->done = 1;
        st->k_done = t;
        atomicOr(&st->err, kErrZeroPivot);
      }
    } else {
      if (threadIdx.x < P) {
        ((T*)a.gi)[threadIdx.x] = G[i * P + threadIdx.x];
        ((T*)a.bj)[threadIdx.x] = Bm[(int64_t)threadIdx.x * m + j];
      }
      if (threadIdx.x == 0) {
        a.col_used[j] = 1;
        a.row_used[i] = 1;
        a.I[t] = i;
        a.J[t] = j;
        if (b.attempts) b.attempts[t] = att + 1;
        st->i = i;
        st->j = j;
        st->a_re = ar;
        st->a_im = ai;
        st->cur = t;
        st->t = t + 1;
        st->fallback = 0;
      }
    }
  } else if (outcome == 2) {
    stop_at(st, t);
  } else if (threadIdx.x == 0) {
    st->fallback = 1;
  }
  if (lead && b.use_graph) cudaGraphSetConditional(b.h_fb, (!st->done && st->fallback) ? 1u : 0u);
}

// Graph mode: whether the step loop runs another iteration.  Every iteration
// draws a pivot or ends the factorization, so at most k + 1 iterations run;
// the iteration count bounds the loop even so.
__global__ void k_bh_ctl(CauchyLikeLaunch a, BhLaunch b) {
  const JobState* st = a.st;
  const int64_t it = ++*b.iter;
  const bool more = !st->done && st->t < a.k && it <= a.k;
  cudaGraphSetConditional(b.h_loop, more ? 1u : 0u);
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
  const unsigned gl = (unsigned)((b.n_sleaf + kGWarps - 1) / kGWarps);
  const unsigned gn = (unsigned)((b.n_sinner + kGWarps - 1) / kGWarps);
  k_bh_gram_leaf<T, P><<<std::max(gl, 1u), kGWarps * 32, 0, s>>>(a, b);
  if (b.n_sinner > 0) k_bh_gram_nodes<P><<<gn, kGWarps * 32, 0, s>>>(a, b);
  if (tm) tm->begin();
  k_bh_bounds<T, P><<<dim3((unsigned)std::max(b.n_tleaf, 1), (unsigned)std::max(b.nslice, 1)), kBThreads, 0, s>>>(a, b);
  if (tm) {
    tm->end();
    tm->all_launches += 2;
  }
}

// The step loop as one CUDA graph: WHILE(h_loop) { Gram passes, bounds, draw,
// IF(h_fb) { exact norms, fallback draw }, update, loop control }.  Captured
// into the conditional bodies on private streams, instantiated and launched
// on s; the graph is freed once its launch completes.
template <typename T, int P>
cudaError_t launch_graph_tp(int32_t dtype, const CauchyLikeLaunch& a, BhLaunch b, cudaStream_t s) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStream_t cs = nullptr, cs2 = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&b.h_loop, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&b.h_fb, g, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking);
  cudaGraphNodeParams wp = {};
  std::memset(static_cast<void*>(&wp), 0, sizeof(wp));
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = b.h_loop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wn = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp);
  b.use_graph = 1;
  bool capturing = false;
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, wp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    capturing = true;
    launch_bounds_tp<T, P>(a, b, cs, nullptr);
    k_bh_sample<T, P><<<kCl, kClThreads, 0, cs>>>(a, b);
    e = cudaGetLastError();
  }
  cudaGraphNodeParams ip = {};
  std::memset(static_cast<void*>(&ip), 0, sizeof(ip));
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = b.h_fb;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  if (e == cudaSuccess) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd);
    cudaGraphNode_t in = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&in, cg, deps, nullptr, nd, &ip);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &in, nullptr, 1, cudaStreamSetCaptureDependencies);
  }
  if (e == cudaSuccess) {
    e = cudaStreamBeginCaptureToGraph(cs2, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      CauchyLikeLaunch forced = a;
      forced.gate = kGateForced;  // the IF node runs only for a pending fallback
      e = cauchy_like_norms(dtype, forced, cs2);
      k_bh_fallback<T, P><<<1, kSThreads, 0, cs2>>>(a, b);
      if (e == cudaSuccess) e = cudaGetLastError();
      cudaGraph_t ig = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(cs2, &ig);
      if (e == cudaSuccess) e = e2;
    }
  }
  if (e == cudaSuccess) {
    e = cauchy_like_update(dtype, a, cs);
    k_bh_ctl<<<1, 1, 0, cs>>>(a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (capturing) {
    cudaGraph_t bg = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &bg);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b.iter, 0, sizeof(int64_t), s);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
  if (ge) cudaGraphExecDestroy(ge);  // freed when the launch completes
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  if (cs2) cudaStreamDestroy(cs2);
  return e;
}

// Without the exact passes: ends the factorization at k when no stop came first.
__global__ void k_bh_end(CauchyLikeLaunch a) {
  JobState* st = a.st;
  if (!st->done) {
    st->done = 1;
    st->k_done = a.k;
  }
}

template <typename T, int P>
cudaError_t run_tp(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm) {
  CauchyLikeLaunch forced = a, gated = a;
  forced.gate = kGateForced;
  gated.gate = kGateFallback;
  cudaError_t e = cudaSuccess;
  if (b.exact_ends) {
    e = cauchy_like_norms(dtype, forced, s);
    if (e != cudaSuccess) return e;
    k_bh_t0<<<1, 1024, 0, s>>>(a);
    tm->all_launches += 3;
  }
  // one graph launch for the whole loop, unless the per-kernel timer is on
  // (events cannot be recorded inside conditional bodies)
  const bool graph = !tm->on && b.iter != nullptr && a.k >= 8;
  if (graph) {
    e = launch_graph_tp<T, P>(dtype, a, b, s);
    if (e != cudaSuccess) return e;
  }
  for (int64_t t = 0; t < (graph ? 0 : a.k); ++t) {
    launch_bounds_tp<T, P>(a, b, s, tm);
    k_bh_sample<T, P><<<kCl, kClThreads, 0, s>>>(a, b);
    e = cauchy_like_norms(dtype, gated, s);
    if (e != cudaSuccess) return e;
    k_bh_fallback<T, P><<<1, kSThreads, 0, s>>>(a, b);
    e = cauchy_like_update(dtype, a, s);
    if (e != cudaSuccess) return e;
    tm->all_launches += 5;
  }
  if (!b.exact_ends) {
    k_bh_end<<<1, 1, 0, s>>>(a);
    tm->all_launches += 1;
    return cudaGetLastError();
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

}  // namespace
}  // namespace rplu
