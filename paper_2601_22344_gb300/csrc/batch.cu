// rplu_batch and the batch plan: many independent small factorizations in one
// persistent launch (off-diagonal Cauchy blocks of a hierarchical matrix,
// Sec. 5.1; dense blocks alike).
//
// k_batch is persistent: each CTA factors one job from its first step to its
// last and then takes the next job from a global counter.  Jobs are visited in
// order of decreasing size, so the largest start first.  A step of a job runs
// entirely inside its CTA (Algorithm 1 with the two-stage draw of Sec. 4.1):
//   row draw by d, pivot row S^(t)(i,:), column draw by its squared entries,
//   then one pass over the job's rows that forms l_p = S^(t)(p,j)/a (FP64
//   division), S^(t+1)(p,:) = S^(t)(p,:) - l_p U(t,:) and d_p = ||S^(t+1)(p,:)||^2.
// Shared memory holds d, the pivot flags, and the pivot rows U(t0..t,:) and
// multipliers L(:,t0..t) of the current block of steps.  The residual itself is
// never written every step: S^(t) = S^(t0) - sum_{s=t0}^{t-1} L(:,s) U(s,:) is
// formed in registers from the block start S^(t0) with the same fused
// multiply-adds, in the same order, as an eager update, and written to the
// job's workspace every `blk` steps.  Before the first write-back S^(0) = A is
// read from the job's input, so a job that stops within blk steps never
// touches a workspace.
//
// Cauchy jobs take the generator form (b_job_gen, Sec. 5.1 with
// displacement rank 1): the residual of A_pq = 1/(x_p - y_q) after any number
// of steps is S_pq = G_p B_q / (x_p - y_q), with generators G (n) and B (m)
// updated in O(n + m) per step (Eqs. generator_update_g / generator_update_b),
// so |S_pq|^2 = |G_p|^2 |B_q|^2 / |x_p - y_q|^2 and each squared row norm is
// |G_p|^2 sum_q w_q / |x_p - y_q|^2 with w_q = |B_q|^2: one reciprocal and a
// few FP32 operations per generated entry, exact norms every step, no
// residual stored and nothing written back, however long the job runs.
//
// The numbers do not depend on the launch shape: the draws are exact
// fixed-point sums (sampler.cuh), the update chain is fixed, and each squared
// row norm is summed per lane over the columns lane, lane+32, ... in order,
// then across lanes by a fixed FP64 tree.  The autotuner may therefore pick
// any shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "batch.h"
#include "cauchy_like.cuh"
#include "common.cuh"
#include "kernels.h"
#include "sampler.cuh"

namespace rplu {
namespace {

template <typename T> struct alignas(16) BVec { T v[Traits<T>::kVec]; };

__device__ __forceinline__ float sq_add(float x, float acc) { return fmaf(x, x, acc); }
__device__ __forceinline__ double sq_add(double x, double acc) { return fma(x, x, acc); }

// Multiplier c / a of the current step.  FP32: the correctly rounded FP32
// quotient, which equals the FP64 quotient rounded to FP32 (double rounding
// through a format of at least 2p + 2 bits is innocuous for division:
// Figueroa, "When is double rounding innocuous?", SIGNUM 1995), so FP32 jobs
// get the FP64-division multiplier without the FP64 pipe.
__device__ __forceinline__ float pivot_div(float c, double a, double) { return __fdiv_rn(c, (float)a); }
__device__ __forceinline__ double pivot_div(double c, double a, double) { return __ddiv_rn(c, a); }
// complex64: the FP64 complex quotient (the dense path's multiplier), rounded to complex64
__device__ __forceinline__ cf32 pivot_div(cf32 c, double ar, double ai) {
  double qr, qi;
  cdiv_d((double)c.re, (double)c.im, ar, ai, qr, qi);
  return cf32{(float)qr, (float)qi};
}

// Loads through L2 only (ld.global.cg), for every element type.
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ cf32 ld_cg(const cf32* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cf32{v.x, v.y};
}

// Squared magnitude accumulated in the real type.
__device__ __forceinline__ float sq_add(cf32 x, float acc) { return fmaf(x.im, x.im, fmaf(x.re, x.re, acc)); }

// v times a 0/1 column mask (exact).
__device__ __forceinline__ float mask_v(float v, float k) { return v * k; }
__device__ __forceinline__ double mask_v(double v, double k) { return v * k; }
__device__ __forceinline__ cf32 mask_v(cf32 v, cf32 k) { return cf32{v.re * k.re, v.im * k.re}; }
__device__ __forceinline__ bool is_zero(float v) { return v == 0.f; }
__device__ __forceinline__ bool is_zero(double v) { return v == 0.0; }
__device__ __forceinline__ bool is_zero(cf32 v) { return v.re == 0.f && v.im == 0.f; }

// Flags raised by the initial pass.
enum : int { kFlagNonFinite = 1, kFlagCancel = 4 };

// Shared-memory carve-up, identical on host and device.
struct BLayout {
  int64_t upend, lpend, d, rused, ckeep, total;
};
__host__ __device__ inline int64_t b_align16(int64_t v) { return (v + 15) / 16 * 16; }
__host__ __device__ inline BLayout b_layout(int64_t n_max, int64_t lds_max, int blk, int w) {
  BLayout L;
  L.upend = 0;
  L.lpend = b_align16(L.upend + (int64_t)blk * lds_max * w);
  L.d = b_align16(L.lpend + (int64_t)blk * n_max * w);
  L.rused = b_align16(L.d + n_max * 8);
  L.ckeep = b_align16(L.rused + n_max);
  L.total = b_align16(L.ckeep + lds_max * w);
  return L;
}

// Generator-form jobs: per column the pair (y_q, w_q = |B_q|^2) read by the
// norm pass, B, the pivot row; per row G, d, and the norm pass's partial sums.
template <typename T> struct GenQ;
template <> struct alignas(8) GenQ<float> { float y, w; };
template <> struct alignas(16) GenQ<double> { double y, w; };
template <> struct alignas(16) GenQ<cf32> { float yr, yi, w, pad; };

struct GLayout {
  int64_t q, b, row, g, d, part, total;  // row and part share one region (never live together)
};
// The norm pass's items (row pairs x column slices): about kGenItems, a
// function of n alone so that every launch shape sums in the same order.
constexpr int64_t kGenItems = 1024;
__host__ __device__ inline int64_t g_items_cap(int64_t n_max) {
  const int64_t half = (n_max + 1) / 2;
  return half > kGenItems ? half : kGenItems;
}
__host__ __device__ inline GLayout g_layout(int64_t n_max, int64_t m_max, int qbytes, int w) {
  GLayout L;
  L.q = 0;
  L.b = b_align16(L.q + m_max * qbytes);
  L.g = b_align16(L.b + m_max * w);
  L.d = b_align16(L.g + n_max * w);
  L.row = L.part = b_align16(L.d + n_max * 8);
  const int64_t row_bytes = m_max * w, part_bytes = g_items_cap(n_max) * 2 * 8;
  L.total = b_align16(L.part + (row_bytes > part_bytes ? row_bytes : part_bytes));
  return L;
}

template <typename T>
struct JobCtx {
  const BatchDesc* jb;
  int64_t n, m, k;
  const T* rows;  // S^(t0): the job's A before the first write-back, then S; row stride ld, 16-byte aligned rows
  int64_t ld;
  T* S;           // workspace (row stride lds)
  int64_t lds;
  T* upend;       // blk x lds_max (row s at upend + s * lds_max)
  T* lpend;       // blk x n_max
  double* d;
  uint8_t* rused;
  T* ckeep;        // 0 for pivoted columns and for the padding q >= m, else 1
  int64_t lds_max, n_max;
};

// Entry (p, q < m) of S^(t0).
// Inputs are read through L2 only (ld.global.cg): in the serving kernel a job's
// buffers may be refilled by copies while the kernel runs, and a stale L1 line
// from an earlier job must not be seen.
template <typename T>
__device__ __forceinline__ T src_at(const JobCtx<T>& c, int64_t p, int64_t q) {
  return ld_cg(c.rows + p * c.ld + q);
}

// Vector g of row p of S^(t0): full (g*W + W <= m) or the ragged last one.
template <typename T, bool kFull>
__device__ __forceinline__ BVec<T> src_vec(const JobCtx<T>& c, int64_t p, int64_t g) {
  constexpr int W = Traits<T>::kVec;
  BVec<T> v;
  if constexpr (kFull) {
    const float4 r = __ldcg(reinterpret_cast<const float4*>(c.rows + p * c.ld + g * W));
    memcpy(&v, &r, 16);
  } else {
#pragma unroll
    for (int e = 0; e < W; ++e) {
      const int64_t q = g * W + e;
      v.v[e] = q < c.m ? src_at(c, p, q) : zero_v<T>();
    }
  }
  return v;
}

// Combine two (hi, lo) FP32 partial sums: TwoSum of the high parts, whose
// rounding error is exact, added to the low parts.  Symmetric in its operands.
__device__ __forceinline__ void pair_add(float& h, float& l, float h2, float l2) {
  const float s = __fadd_rn(h, h2);
  const float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
  h = s;
  l = __fadd_rn(__fadd_rn(l, l2), e);
}
__device__ __forceinline__ void pair_add(double& h, double& l, double h2, double l2) {
  h += h2;
  (void)l;
  (void)l2;
}

// Rows are processed by 8-lane segments: lane sl of a segment visits the
// column vectors sl, sl + 8, sl + 16, ... of its row(s), and the segment's
// per-lane FP32 partial sums are combined by the fixed tree xor 4, 2, 1 on
// (hi, lo) pairs (pair_add).  The four segments of a warp read the same
// column vectors, so loads of the column mask and the pivot rows are
// broadcasts.  The tree does not depend on how many rows a lane carries or
// on the block size.
constexpr int kSeg = 8;

template <typename real>
__device__ __forceinline__ void seg_sum(real acc, real& h, real& l) {
  h = acc;
  l = 0;
#pragma unroll
  for (int o = kSeg / 2; o > 0; o >>= 1) {
    const real rh = __shfl_xor_sync(0xffffffffu, h, o), rl = __shfl_xor_sync(0xffffffffu, l, o);
    pair_add(h, l, rh, rl);
  }
}

// Multipliers of step t (pivot column j, pivot value a, r pending steps):
// l_p = S^(t)(p, j) / a for unpivoted rows, one row per thread, into lpend[r]
// and L(:,t); L(p,t) = 1 on the pivot row and 0 on earlier pivot rows.
template <typename T>
__device__ void b_multipliers(const JobCtx<T>& c, int r, int64_t t, int64_t i, int64_t j, double ar, double ai) {
  T* Lout = (T*)c.jb->L;
  for (int64_t p = threadIdx.x; p < c.n; p += blockDim.x) {
    if (c.rused[p]) {
      Lout[t * c.n + p] = p == i ? one_v<T>() : zero_v<T>();
      continue;
    }
    T v = src_at(c, p, j);
    for (int s = 0; s < r; ++s) v = fms(v, c.lpend[(int64_t)s * c.n_max + p], c.upend[(int64_t)s * c.lds_max + j]);
    const T l = pivot_div(v, ar, ai);
    c.lpend[(int64_t)r * c.n_max + p] = l;
    Lout[t * c.n + p] = l;
  }
}

// One pass over the job's rows applying NP updates (the pending steps of the
// block plus the current one, whose multipliers are in lpend; 0 for the
// initial norms): S^(t+1)(p,:) in registers, d_p = its squared norm over the
// kept columns.  A warp takes 4 * RL rows at a time (RL per lane).  wb: write
// S^(t+1) to the workspace.  check: flag non-finite entries.
template <typename T, int NT, int RL, int NP>
__device__ void b_pass(const JobCtx<T>& c, bool wb, bool check, int* flags) {
  using real = typename Traits<T>::real;
  constexpr int W = Traits<T>::kVec;
  constexpr int NW = NT / 32;
  constexpr int RPW = (32 / kSeg) * RL;  // rows per warp tile
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = lane / kSeg, sl = lane % kSeg;
  const int64_t ngrp = (c.m + W - 1) / W, nfull = c.m / W;
  bool badl = false;
  for (int64_t p0 = (int64_t)warp * RPW; p0 < c.n; p0 += (int64_t)NW * RPW) {
    bool on[RL];
    int64_t pr[RL];  // row read (clamped into range; results of rows that are off are discarded)
    bool any = false;
#pragma unroll
    for (int k = 0; k < RL; ++k) {
      const int64_t p = p0 + seg * RL + k;
      on[k] = p < c.n && !c.rused[p];
      pr[k] = p < c.n ? p : c.n - 1;
      any |= on[k];
    }
    if (!__any_sync(0xffffffffu, any)) continue;
    T lm[RL][NP > 0 ? NP : 1];
#pragma unroll
    for (int k = 0; k < RL; ++k) {
#pragma unroll
      for (int s = 0; s < NP; ++s) lm[k][s] = on[k] ? c.lpend[(int64_t)s * c.n_max + pr[k]] : zero_v<T>();
    }
    real acc[RL];
#pragma unroll
    for (int k = 0; k < RL; ++k) acc[k] = 0;
    // one column vector g of this lane's rows, given its S^(t0) values v
    auto update = [&](int64_t g, BVec<T>(&v)[RL], auto full) {
      constexpr bool kFull = decltype(full)::value;
      if (check) {
#pragma unroll
        for (int k = 0; k < RL; ++k)
#pragma unroll
          for (int e = 0; e < W; ++e) {
            const bool real_entry = on[k] && (kFull || g * W + e < c.m);
            badl |= real_entry && !finite_v(v[k].v[e]);
          }
      }
      if constexpr (NP > 0) {
#pragma unroll
        for (int s = 0; s < NP; ++s) {
          const float4 ur = *reinterpret_cast<const float4*>(c.upend + (int64_t)s * c.lds_max + g * W);
          BVec<T> u;
          memcpy(&u, &ur, 16);
#pragma unroll
          for (int k = 0; k < RL; ++k)
#pragma unroll
            for (int e = 0; e < W; ++e) v[k].v[e] = fms(v[k].v[e], lm[k][s], u.v[e]);
        }
      }
      // squares of the kept columns: multiplying by the 0/1 mask is exact
      const float4 kr = *reinterpret_cast<const float4*>(c.ckeep + g * W);
      BVec<T> keep;
      memcpy(&keep, &kr, 16);
#pragma unroll
      for (int e = 0; e < W; ++e)
#pragma unroll
        for (int k = 0; k < RL; ++k) {
          const T vm = mask_v(v[k].v[e], keep.v[e]);
          acc[k] = sq_add(vm, acc[k]);
        }
      if (wb) {
#pragma unroll
        for (int k = 0; k < RL; ++k)
          if (on[k]) {
            float4 o;
            memcpy(&o, &v[k], 16);
            *reinterpret_cast<float4*>(c.S + pr[k] * c.lds + g * W) = o;
          }
      }
    };
    int64_t g = sl;
    {
      // issue the loads of 4 vectors (kUnr column vectors of RL rows) before using any,
      // so that a CTA keeps enough bytes in flight (the per-lane order of the
      // updates and of the squared-norm sum is unchanged)
      constexpr int kUnr = 4 / RL;
      for (; g + (kUnr - 1) * kSeg < nfull; g += kUnr * kSeg) {
        BVec<T> v[kUnr][RL];
#pragma unroll
        for (int u = 0; u < kUnr; ++u)
#pragma unroll
          for (int k = 0; k < RL; ++k) v[u][k] = src_vec<T, true>(c, pr[k], g + u * kSeg);
#pragma unroll
        for (int u = 0; u < kUnr; ++u) update(g + u * kSeg, v[u], std::true_type{});
      }
    }
    for (; g < ngrp; g += kSeg) {
      BVec<T> v[RL];
      if (g < nfull) {
#pragma unroll
        for (int k = 0; k < RL; ++k) v[k] = src_vec<T, true>(c, pr[k], g);
        update(g, v, std::true_type{});
      } else {
#pragma unroll
        for (int k = 0; k < RL; ++k) v[k] = src_vec<T, false>(c, pr[k], g);
        update(g, v, std::false_type{});
      }
    }
#pragma unroll
    for (int k = 0; k < RL; ++k) {
      real h, l;
      seg_sum(acc[k], h, l);
      if (sl == 0 && on[k]) c.d[pr[k]] = (double)h + (double)l;  // one FP64 combine, on the writer lane
    }
  }
  if (check) {
    const bool b1 = __any_sync(0xffffffffu, badl);
    if (lane == 0 && b1) atomicOr(flags, kFlagNonFinite);
  }
}

// The pass for a run-time number of updates np (0..8, the largest write-back interval).
template <typename T, int NT, int RL>
__device__ void b_pass_rt(const JobCtx<T>& c, int np, bool wb, bool check, int* flags) {
  switch (np) {
    case 0: b_pass<T, NT, RL, 0>(c, wb, check, flags); break;
    case 1: b_pass<T, NT, RL, 1>(c, wb, check, flags); break;
    case 2: b_pass<T, NT, RL, 2>(c, wb, check, flags); break;
    case 3: b_pass<T, NT, RL, 3>(c, wb, check, flags); break;
    case 4: b_pass<T, NT, RL, 4>(c, wb, check, flags); break;
    case 5: b_pass<T, NT, RL, 5>(c, wb, check, flags); break;
    case 6: b_pass<T, NT, RL, 6>(c, wb, check, flags); break;
    case 7: b_pass<T, NT, RL, 7>(c, wb, check, flags); break;
    default: b_pass<T, NT, RL, 8>(c, wb, check, flags); break;
  }
}

template <typename T, int NT, int R>
__device__ void b_job(BatchDesc* jbp, const BatchArgs& a, unsigned char* smem, FxScratch& sh, int* s_bad,
                      const volatile int32_t* cancel = nullptr) {
  constexpr int W = Traits<T>::kVec;
  const BatchDesc& jb = *jbp;
  const int tid = threadIdx.x;
  const BLayout Ly = b_layout(a.n_max, a.lds_max, a.blk, (int)sizeof(T));
  JobCtx<T> c;
  c.jb = jbp;
  c.n = jb.n;
  c.m = jb.m;
  c.k = jb.k_max;
  c.rows = (const T*)jb.A;
  c.ld = jb.lda;
  c.S = (T*)jb.S;
  c.lds = jb.lds;
  c.upend = (T*)(smem + Ly.upend);
  c.lpend = (T*)(smem + Ly.lpend);
  c.d = (double*)(smem + Ly.d);
  c.rused = smem + Ly.rused;
  c.ckeep = (T*)(smem + Ly.ckeep);
  c.lds_max = a.lds_max;
  c.n_max = a.n_max;
  const int64_t ldsj = (c.m + W - 1) / W * W;  // padded row length of this job in the shared buffers

  for (int64_t p = tid; p < c.n; p += NT) c.rused[p] = 0;
  for (int64_t q = tid; q < ldsj; q += NT) c.ckeep[q] = q < c.m ? one_v<T>() : zero_v<T>();
  for (int64_t s = tid; s < (int64_t)a.blk * ldsj; s += NT) {
    const int64_t r = s / ldsj, q = s - r * ldsj;
    c.upend[r * c.lds_max + q] = zero_v<T>();
  }
  if (tid == 0) *s_bad = 0;
  __syncthreads();

  // initial squared row norms (a1), checking every entry
  b_pass_rt<T, NT, R>(c, 0, false, true, s_bad);
  __syncthreads();
  int32_t err = (*s_bad & kFlagNonFinite) ? kErrNonFinite : 0;
  int64_t t = 0, t0 = 0;
  double T0 = 0.0, Tlast = 0.0;
  bool stopped = err != 0;
  if (!stopped) {
    for (; t < c.k; ++t) {
      const int r = (int)(t - t0);
      if (cancel) {
        // serving: the caller may cancel a running job between steps
        if (tid == 0) *s_bad = *cancel ? kFlagCancel : 0;
        __syncthreads();
        if (*s_bad & kFlagCancel) {
          err = kErrCancelled;
          break;
        }
      }
      uint64_t mb = 0;
      for (int64_t p = tid; p < c.n; p += NT) {
        const uint64_t b = fx_bits64(c.d[p]);
        mb = b > mb ? b : mb;
      }
      mb = block_max_u64(mb, sh);
      const int Er = fx_scale_f64(mb, c.n);
      const double* dd = c.d;
      auto dw = [dd, Er](int64_t p) -> u128 { return fx_f64(dd[p], Er); };
      int64_t i = -1, j = -1;
      bool ok = false;
      T* rh = c.upend + (int64_t)r * c.lds_max;
      T* Urow = (T*)jb.U + t * c.m;
      for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
        u128 Tfx;
        if (a.mode == RPLU_PIVOT_RANDOM) {
          i = fx_block_draw(dw, c.n, draw_u53(jb.seed, t, 0, attempt), true, &Tfx, sh);
        } else {
          (void)fx_block_draw(dw, c.n, 0, false, &Tfx, sh);
          i = fx_block_argmax([dd](int64_t p) -> uint64_t { return fx_bits64(dd[p]); }, c.n, sh);
        }
        const double Tt = fx_to_double(Tfx, Er);
        if (attempt == 0) {
          if (t == 0) T0 = Tt;
          Tlast = Tt;
          if (!(Tt > 0.0) || (jb.tol > 0.0 && Tt <= jb.tol * jb.tol * T0)) break;
        } else if (!(Tt > 0.0)) {
          break;
        }
        if (i < 0) break;
        // S^(t)(i,:): S^(t0)(i,:) minus the pending updates, pivoted columns masked
        uint64_t cb = 0;
        for (int64_t q = tid; q < ldsj; q += NT) {
          T v = q < c.m ? src_at(c, i, q) : zero_v<T>();
          for (int s = 0; s < r; ++s)
            v = fms(v, c.lpend[(int64_t)s * c.n_max + i], c.upend[(int64_t)s * c.lds_max + q]);
          v = is_zero(c.ckeep[q]) ? zero_v<T>() : v;
          rh[q] = v;
          if (q < c.m) Urow[q] = v;
          const uint64_t b = entry_max_bits(v);
          cb = b > cb ? b : cb;
        }
        cb = block_max_u64(cb, sh);  // also orders the row writes before the reads below
        const int Ec = fx_entry_scale<T>(cb, c.m);
        const T* rr = rh;
        auto cw = [rr, Ec](int64_t q) -> u128 { return fx_abs2(rr[q], Ec); };
        u128 Rfx = 1;
        if (a.mode == RPLU_PIVOT_RANDOM) {
          j = fx_block_draw(cw, c.m, draw_u53(jb.seed, t, 1, attempt), true, &Rfx, sh);
        } else {
          (void)fx_block_draw(cw, c.m, 0, false, &Rfx, sh);
          j = fx_block_argmax(cw, c.m, sh);
        }
        if (Rfx == 0 || j < 0) {
          if (tid == 0) c.d[i] = 0.0;
          __syncthreads();
          continue;
        }
        ok = true;
        break;
      }
      if (!ok) break;
      double ap, api;
      to_d(rh[j], ap, api);
      __syncthreads();
      if (tid == 0) {
        c.rused[i] = 1;
        c.ckeep[j] = zero_v<T>();
        c.d[i] = 0.0;
        jb.I[t] = i;
        jb.J[t] = j;
      }
      __syncthreads();
      const bool wb = (r + 1 == a.blk) && (t + 1 < c.k) && c.S != nullptr;
      b_multipliers(c, r, t, i, j, ap, api);
      __syncthreads();
      b_pass_rt<T, NT, R>(c, r + 1, wb, false, s_bad);
      __syncthreads();
      if (wb) {
        t0 = t + 1;
        c.rows = c.S;
        c.ld = c.lds;
      }
    }
    if (t == c.k) {
      // ||S||_F^2 after the last step
      uint64_t mb = 0;
      for (int64_t p = tid; p < c.n; p += NT) {
        const uint64_t b = fx_bits64(c.d[p]);
        mb = b > mb ? b : mb;
      }
      mb = block_max_u64(mb, sh);
      const int Er = fx_scale_f64(mb, c.n);
      const double* dd = c.d;
      u128 Tfx;
      (void)fx_block_draw([dd, Er](int64_t p) -> u128 { return fx_f64(dd[p], Er); }, c.n, 0, false, &Tfx, sh);
      Tlast = fx_to_double(Tfx, Er);
      if (c.k == 0) T0 = Tlast;
    }
  }
  for (int64_t s = t + tid; s < c.k; s += NT) {
    jb.I[s] = -1;
    jb.J[s] = -1;
  }
  if (tid == 0) {
    jbp->k_done = err ? 0 : t;
    jbp->T0 = T0;
    jbp->T_final = Tlast;
    jbp->err = err;
  }
}

// ----------------------------------------------------------- generator form
// A Cauchy job in the generator form (see the top of the file): per step the
// exact squared row norms from the generators, the row draw, the pivot row
// r_q = G_i B_q / (x_i - y_q), the column draw, the pivot column, the
// multipliers l_p = c_p / a (FP64 division), U(t,:) = r, L(:,t) = l, and the
// generator updates G <- G - l G_i, B <- B - B_j (r / a) with the pivot's G_i
// and B_j set to exact zero (so pivoted rows and columns weigh exactly 0 in
// every later draw).  The norm pass splits the rows into pairs and the columns
// into S slices, about kGenItems (pair, slice) items;
// each item sums its slice in the working precision, folding into FP64 every
// 64 columns; a row's slices are added in slice order.
__device__ __forceinline__ float w_of(float b) { return b * b; }
__device__ __forceinline__ double w_of(double b) { return b * b; }
__device__ __forceinline__ float w_of(cf32 b) { return fmaf(b.re, b.re, b.im * b.im); }
__device__ __forceinline__ GenQ<float> make_q(float y, float w) { return GenQ<float>{y, w}; }
__device__ __forceinline__ GenQ<double> make_q(double y, double w) { return GenQ<double>{y, w}; }
__device__ __forceinline__ GenQ<cf32> make_q(cf32 y, float w) { return GenQ<cf32>{y.re, y.im, w, 0.f}; }
// w / |x - y|^2 with the hardware reciprocal (FP32) or an FP64 division
__device__ __forceinline__ float inv_sq(float x, const GenQ<float>& q) {
  const float z = x - q.y;
  return q.w * rcp_fast(z * z);
}
__device__ __forceinline__ double inv_sq(double x, const GenQ<double>& q) {
  const double z = x - q.y;
  return q.w / (z * z);
}
__device__ __forceinline__ float inv_sq(cf32 x, const GenQ<cf32>& q) {
  const float zr = x.re - q.yr, zi = x.im - q.yi;
  return q.w * rcp_fast(fmaf(zr, zr, zi * zi));
}

// q / a for the multipliers and the B update: the FP64 quotient rounded to
// the working precision.  Real FP32 data divide in FP32 with correct rounding,
// which gives the same bits (double rounding through binary64 is innocuous for
// division: Figueroa 1995) without the FP64 pipe; the other types use cdiv_d.
template <typename T>
__device__ __forceinline__ T quot(T q, double ar, double ai) {
  if constexpr (std::is_same<T, float>::value) {
    return __fdiv_rn(q, (float)ar);
  } else {
    double qr, qi, lr, li;
    to_d(q, qr, qi);
    cdiv_d(qr, qi, ar, ai, lr, li);
    return from_d<T>(lr, li);
  }
}

template <typename T, int NT>
__device__ void b_job_gen(BatchDesc* jbp, const BatchArgs& a, unsigned char* smem, FxScratch& sh,
                          const volatile int32_t* cancel = nullptr) {
  using real = typename Traits<T>::real;
  const BatchDesc& jb = *jbp;
  const int tid = threadIdx.x;
  const int64_t n = jb.n, m = jb.m, kmax = jb.k_max;
  const GLayout Ly = g_layout(a.gn_max, a.gm_max, (int)sizeof(GenQ<T>), (int)sizeof(T));
  GenQ<T>* qv = (GenQ<T>*)(smem + Ly.q);
  T* Bg = (T*)(smem + Ly.b);
  T* row = (T*)(smem + Ly.row);
  T* Gg = (T*)(smem + Ly.g);
  double* d = (double*)(smem + Ly.d);
  double* part = (double*)(smem + Ly.part);
  __shared__ int s_flag;
  const T* xg = (const T*)jb.x;
  const T* yg = (const T*)jb.y;
  T* Lout = (T*)jb.L;

  for (int64_t q = tid; q < m; q += NT) {
    const T yq = ld_cg(yg + q);
    Bg[q] = one_v<T>();
    qv[q] = make_q(yq, (real)1);
  }
  for (int64_t p = tid; p < n; p += NT) Gg[p] = one_v<T>();
  if (tid == 0) s_flag = 0;
  __syncthreads();

  // the norm pass's split: pairs of rows x S column slices, about kGenItems items
  const int64_t pairs = (n + 1) / 2;
  int64_t S = pairs > 0 ? kGenItems / pairs : 1;
  S = S < 1 ? 1 : (S > 32 ? 32 : S);
  if (S > m) S = m > 0 ? m : 1;
  const int64_t items = pairs * S;
  const int64_t qlen = (m + S - 1) / S;

  // d_p = |G_p|^2 sum_q w_q / |x_p - y_q|^2; flags a non-finite norm
  auto norms = [&]() {
    bool bad = false;
    for (int64_t it = tid; it < items; it += NT) {
      const int64_t sl = it / pairs, pr = it - sl * pairs;
      const int64_t p0 = 2 * pr, p1 = p0 + 1;
      const bool on0 = w_of(Gg[p0]) != (real)0, on1 = p1 < n && w_of(Gg[p1]) != (real)0;
      double s0 = 0.0, s1 = 0.0;
      if (on0 || on1) {
        const T x0 = ld_cg(xg + p0), x1 = p1 < n ? ld_cg(xg + p1) : x0;
        const int64_t q0 = sl * qlen, q1 = min(m, q0 + qlen);
        for (int64_t c0 = q0; c0 < q1; c0 += 64) {
          const int64_t c1 = min(q1, c0 + 64);
          real a0 = 0, a1 = 0;
          for (int64_t q = c0; q < c1; ++q) {
            const GenQ<T> e = qv[q];
            a0 += inv_sq(x0, e);
            a1 += inv_sq(x1, e);
          }
          s0 += (double)a0;
          s1 += (double)a1;
        }
      }
      part[2 * it] = on0 ? s0 : 0.0;
      part[2 * it + 1] = on1 ? s1 : 0.0;
    }
    __syncthreads();
    for (int64_t p = tid; p < n; p += NT) {
      const int64_t pr = p >> 1, r = p & 1;
      double acc = 0.0;
      for (int64_t sl = 0; sl < S; ++sl) acc += part[2 * (sl * pairs + pr) + r];
      const double v = (double)w_of(Gg[p]) * acc;
      bad |= !isfinite(v);
      d[p] = v;
    }
    if (__syncthreads_or(bad) && tid == 0) s_flag = 1;
    __syncthreads();
  };

  norms();
  int32_t err = s_flag ? kErrNonFinite : 0;
  int64_t t = 0;
  double T0 = 0.0, Tlast = 0.0;
  if (!err) {
    for (; t < kmax; ++t) {
      if (cancel) {
        if (tid == 0) s_flag = *cancel ? 2 : 0;
        __syncthreads();
        if (s_flag == 2) {
          err = kErrCancelled;
          break;
        }
      }
      uint64_t mb = 0;
      for (int64_t p = tid; p < n; p += NT) {
        const uint64_t b = fx_bits64(d[p]);
        mb = b > mb ? b : mb;
      }
      mb = block_max_u64(mb, sh);
      const int Er = fx_scale_f64(mb, n);
      const double* dd = d;
      auto dw = [dd, Er](int64_t p) -> u128 { return fx_f64(dd[p], Er); };
      int64_t i = -1, j = -1;
      bool ok = false;
      T* Urow = (T*)jb.U + t * m;
      for (int attempt = 0; attempt < kMaxAttempts; ++attempt) {
        u128 Tfx;
        if (a.mode == RPLU_PIVOT_RANDOM) {
          i = fx_block_draw(dw, n, draw_u53(jb.seed, t, 0, attempt), true, &Tfx, sh);
        } else {
          (void)fx_block_draw(dw, n, 0, false, &Tfx, sh);
          i = fx_block_argmax([dd](int64_t p) -> uint64_t { return fx_bits64(dd[p]); }, n, sh);
        }
        const double Tt = fx_to_double(Tfx, Er);
        if (attempt == 0) {
          if (t == 0) T0 = Tt;
          Tlast = Tt;
          if (!(Tt > 0.0) || (jb.tol > 0.0 && Tt <= jb.tol * jb.tol * T0)) break;
        } else if (!(Tt > 0.0)) {
          break;
        }
        if (i < 0) break;
        // pivot row r_q = G_i B_q / (x_i - y_q): zero on pivoted columns (B_q = 0)
        const T gi = Gg[i];
        const T xi = ld_cg(xg + i);
        uint64_t cb = 0;
        for (int64_t q = tid; q < m; q += NT) {
          const T v = div_v(mul_v(gi, Bg[q]), sub_v(xi, ld_cg(yg + q)));
          row[q] = v;
          Urow[q] = v;
          const uint64_t b = entry_max_bits(v);
          cb = b > cb ? b : cb;
        }
        cb = block_max_u64(cb, sh);  // also orders the row writes before the reads below
        const int Ec = fx_entry_scale<T>(cb, m);
        const T* rr = row;
        auto cw = [rr, Ec](int64_t q) -> u128 { return fx_abs2(rr[q], Ec); };
        u128 Rfx = 1;
        if (a.mode == RPLU_PIVOT_RANDOM) {
          j = fx_block_draw(cw, m, draw_u53(jb.seed, t, 1, attempt), true, &Rfx, sh);
        } else {
          (void)fx_block_draw(cw, m, 0, false, &Rfx, sh);
          j = fx_block_argmax(cw, m, sh);
        }
        if (Rfx == 0 || j < 0) {
          if (tid == 0) d[i] = 0.0;
          __syncthreads();
          continue;
        }
        ok = true;
        break;
      }
      if (!ok) break;
      double ar, ai;
      to_d(row[j], ar, ai);
      const T gi = Gg[i], bj = Bg[j];
      const T yj = ld_cg(yg + j);
      if (tid == 0) {
        jb.I[t] = i;
        jb.J[t] = j;
      }
      __syncthreads();
      // multipliers l_p = c_p / a with c_p = G_p B_j / (x_p - y_j); G <- G - l G_i
      for (int64_t p = tid; p < n; p += NT) {
        T l;
        if (p == i) {
          l = one_v<T>();
          Gg[p] = zero_v<T>();
        } else if (w_of(Gg[p]) == (real)0) {
          l = zero_v<T>();
        } else {
          const T gp = Gg[p];
          l = quot(div_v(mul_v(gp, bj), sub_v(ld_cg(xg + p), yj)), ar, ai);
          Gg[p] = sub_v(gp, mul_v(l, gi));
        }
        Lout[t * n + p] = l;
      }
      // B <- B - B_j (r / a), B_j = 0
      for (int64_t q = tid; q < m; q += NT) {
        T bq;
        if (q == j) {
          bq = zero_v<T>();
        } else {
          bq = sub_v(Bg[q], mul_v(bj, quot(row[q], ar, ai)));
        }
        Bg[q] = bq;
        qv[q].w = w_of(bq);
      }
      __syncthreads();
      norms();
      if (s_flag) {
        err = kErrNonFinite;
        ++t;
        break;
      }
    }
    if (t == kmax && !err) {
      // ||S||_F^2 after the last step
      uint64_t mb = 0;
      for (int64_t p = tid; p < n; p += NT) {
        const uint64_t b = fx_bits64(d[p]);
        mb = b > mb ? b : mb;
      }
      mb = block_max_u64(mb, sh);
      const int Er = fx_scale_f64(mb, n);
      const double* dd = d;
      u128 Tfx;
      (void)fx_block_draw([dd, Er](int64_t p) -> u128 { return fx_f64(dd[p], Er); }, n, 0, false, &Tfx, sh);
      Tlast = fx_to_double(Tfx, Er);
      if (kmax == 0) T0 = Tlast;
    }
  }
  for (int64_t s2 = t + tid; s2 < kmax; s2 += NT) {
    jb.I[s2] = -1;
    jb.J[s2] = -1;
  }
  if (tid == 0) {
    jbp->k_done = err ? 0 : t;
    jbp->T0 = T0;
    jbp->T_final = Tlast;
    jbp->err = err;
  }
}

// FP32 kernels are register-capped for three (256 threads) or six (128
// threads) CTAs per SM, complex64 ones for two; the FP64 one is not capped.
template <typename T, int NT>
constexpr int batch_min_blocks() {
  return Traits<T>::kComplex ? 2 : std::is_same<T, float>::value ? (NT == 256 ? 3 : 6) : 1;
}

template <typename T, int NT, int R>
__global__ void __launch_bounds__(NT, batch_min_blocks<T, NT>()) k_batch(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ FxScratch sh;
  __shared__ int s_job;
  __shared__ int s_bad;
  for (;;) {
    if (threadIdx.x == 0) s_job = atomicAdd(a.counter, 1);
    __syncthreads();
    const int b = s_job;
    if (b >= a.njobs) break;
    BatchDesc* jp = a.jobs + a.order[b];
    if (jp->kind == 1) b_job_gen<T, NT>(jp, a, smem, sh);
    else b_job<T, NT, R>(jp, a, smem, sh, &s_bad);
    __syncthreads();
  }
}

// Serving: a persistent kernel fed by a ring of job descriptors in
// host-mapped memory.  A CTA claims the next published ticket (compare-and-
// swap on the device head, so nothing is claimed before it is published),
// marks it claimed for the host, copies the descriptor to shared memory,
// factors the job exactly as k_batch does for its type and kind (FP32 or
// complex64; dense, or Cauchy in the generator form), writes the results back
// to the ring slot and then, after a system-scope fence, the slot's completion
// sequence.  One kernel serves every type, so requests are taken strictly in
// arrival order and no type waits for SMs held by another.  A CTA that finds
// no ticket for `idle_cycles` SM clocks (or sees the stop flag) exits and says
// so in its `exited` flag; the host launches new CTAs (another launch, on
// another stream) when published tickets stay unclaimed while CTAs have
// exited.  Every wait is bounded.
constexpr int kServeThreads = 256;

template <int NT>
__global__ void __launch_bounds__(NT, 1) k_serve(BatchArgs a, ServeRing q) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ FxScratch sh;
  __shared__ BatchDesc s_desc;
  __shared__ long long s_ticket;
  __shared__ int s_bad;
  for (;;) {
    if (threadIdx.x == 0) {
      long long claimed = -1;
      const long long t0 = clock64();
      unsigned back = 256;  // ns between polls of the host-written tail, doubling to 8 us
      while (!*q.stop) {
        const long long h = (long long)atomicAdd((unsigned long long*)q.head, 0ull);
        long long tl;
        asm volatile("ld.acquire.sys.global.s64 %0, [%1];" : "=l"(tl) : "l"(q.tail) : "memory");
        if (h < tl) {
          if ((long long)atomicCAS((unsigned long long*)q.head, (unsigned long long)h, (unsigned long long)(h + 1)) == h) {
            claimed = h;
            break;
          }
          continue;
        }
        if (clock64() - t0 > q.idle_cycles) break;
        __nanosleep(back);
        back = back < 8192 ? 2 * back : back;
      }
      s_ticket = claimed;
      if (claimed >= 0) {
        q.claimed[claimed % q.cap] = claimed + 1;  // tells the host that a CTA has this ticket
        __threadfence_system();
        const volatile BatchDesc* src = q.desc + claimed % q.cap;
        const volatile uint32_t* w = (const volatile uint32_t*)src;
        uint32_t* d = (uint32_t*)&s_desc;
        for (int k = 0; k < (int)(sizeof(BatchDesc) / 4); ++k) d[k] = w[k];
      }
    }
    __syncthreads();
    const long long h = s_ticket;
    if (h < 0) {
      if (threadIdx.x == 0) {
        __threadfence_system();
        q.exited[blockIdx.x] = 1;  // the host may now launch a CTA in this one's place
      }
      break;
    }
    const int64_t slot = h % q.cap;
    const volatile int32_t* cancel = q.cancel + slot;
    if (s_desc.dtype == RPLU_C64) {
      if (s_desc.kind == 1) b_job_gen<cf32, NT>(&s_desc, a, smem, sh, cancel);
      else b_job<cf32, NT, 1>(&s_desc, a, smem, sh, &s_bad, cancel);
    } else {
      if (s_desc.kind == 1) b_job_gen<float, NT>(&s_desc, a, smem, sh, cancel);
      else b_job<float, NT, 2>(&s_desc, a, smem, sh, &s_bad, cancel);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      volatile BatchDesc* dst = q.desc + slot;
      dst->k_done = s_desc.k_done;
      dst->T0 = s_desc.T0;
      dst->T_final = s_desc.T_final;
      dst->err = s_desc.err;
      __threadfence_system();
      q.done[slot] = (int64_t)(h + 1);
    }
    __syncthreads();
  }
}

template <typename T, int NT, int R>
cudaError_t launch_t(const BatchArgs& a, const BatchShape& sh, int64_t smem, cudaStream_t s) {
  k_batch<T, NT, R><<<sh.grid, NT, (size_t)smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int NT, int R>
cudaError_t occupancy_t(int64_t smem, int* blocks) {
  auto k = k_batch<T, NT, R>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, NT, (size_t)smem);
}

// Compiled shapes: threads per CTA x rows per warp tile (4 rows: one per
// 8-lane segment; 8 rows: two per segment).
#define RPLU_BATCH_DISPATCH(FN, ...)                                               \
  do {                                                                             \
    if (dtype == RPLU_F32) {                                                       \
      if (threads == 128 && rows == 4) return FN<float, 128, 1>(__VA_ARGS__);      \
      if (threads == 128 && rows == 8) return FN<float, 128, 2>(__VA_ARGS__);      \
      if (threads == 256 && rows == 4) return FN<float, 256, 1>(__VA_ARGS__);      \
      if (threads == 256 && rows == 8) return FN<float, 256, 2>(__VA_ARGS__);      \
    } else if (dtype == RPLU_F64) {                                                \
      if (threads == 256 && rows == 8) return FN<double, 256, 2>(__VA_ARGS__);     \
    } else if (dtype == RPLU_C64) {                                                \
      if (threads == 256 && rows == 4) return FN<cf32, 256, 1>(__VA_ARGS__);       \
      if (threads == 256 && rows == 8) return FN<cf32, 256, 2>(__VA_ARGS__);       \
    }                                                                              \
    return cudaErrorInvalidValue;                                                  \
  } while (0)

}  // namespace

int64_t batch_smem_bytes(int32_t dtype, const BatchArgs& a) {
  const int w = dtype == RPLU_F32 ? 4 : 8;
  const int qb = dtype == RPLU_F32 ? 8 : 16;
  int64_t bytes = 0;
  if (a.kinds & kKindDense) bytes = b_layout(a.n_max, a.lds_max, a.blk, w).total;
  if (a.kinds & kKindCauchy) {
    const int64_t g = g_layout(a.gn_max, a.gm_max, qb, w).total;
    bytes = g > bytes ? g : bytes;
  }
  return bytes;
}

int64_t serve_smem_bytes(const BatchArgs& a) {
  const int64_t f = batch_smem_bytes(RPLU_F32, a), c = batch_smem_bytes(RPLU_C64, a);
  return f > c ? f : c;
}

cudaError_t batch_occupancy(int32_t dtype, int threads, int rows, int64_t smem, int* blocks) {
  RPLU_BATCH_DISPATCH(occupancy_t, smem, blocks);
}

cudaError_t serve_occupancy(int64_t smem, int* blocks) {
  auto k = k_serve<kServeThreads>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kServeThreads, (size_t)smem);
}

cudaError_t serve_launch(const BatchArgs& a, const ServeRing& q, int grid, cudaStream_t s) {
  const int64_t smem = serve_smem_bytes(a);
  auto k = k_serve<kServeThreads>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kServeThreads, (size_t)smem, s>>>(a, q);
  return cudaGetLastError();
}

cudaError_t batch_launch(int32_t dtype, const BatchArgs& a, const BatchShape& sh, cudaStream_t s) {
  const int threads = sh.threads, rows = sh.rows;
  const int64_t smem = batch_smem_bytes(dtype, a);
  RPLU_BATCH_DISPATCH(launch_t, a, sh, smem, s);
}

}  // namespace rplu
