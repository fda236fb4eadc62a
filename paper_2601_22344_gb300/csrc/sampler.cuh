// Block-level exact inverse-CDF draw and arg-max over fixed-point weights
// (fixedpoint.h).  Used by the two-stage pivot draw of both forms: a row by
// its squared norm, then a column by the squared entries of that row (paper
// Sec. 4.1).
//
// Layout: warp w of the block owns the contiguous index segment
// [w*seg, (w+1)*seg); lanes read it with stride 32 (coalesced).  Pass 1 sums
// each segment exactly, one thread scans the (at most 32) segment totals, and
// the single warp whose segment holds the target walks it 32 entries at a time
// with a warp prefix scan.  All sums are exact integers, so the drawn index is
// the smallest p with (w_0 + ... + w_p) > floor(U * T / 2^53) for any
// partition of the work.
#pragma once

#include "common.cuh"
#include "fixedpoint.h"

namespace rplu {

struct FxScratch {
  u128 tot[32];
  u128 base[32];
  u128 T;
  u128 target;
  uint64_t key[32];
  int64_t idx[32];
  int64_t found;
  int32_t wstar;
};

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o) {
  const uint64_t lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)v, o);
  const uint64_t hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)(v >> 64), o);
  return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u128 shfl_up_u128(u128 v, int o) {
  const uint64_t lo = __shfl_up_sync(0xffffffffu, (unsigned long long)(uint64_t)v, o);
  const uint64_t hi = __shfl_up_sync(0xffffffffu, (unsigned long long)(uint64_t)(v >> 64), o);
  return ((u128)hi << 64) | lo;
}
__device__ __forceinline__ u128 shfl_idx_u128(u128 v, int src) {
  const uint64_t lo = __shfl_sync(0xffffffffu, (unsigned long long)(uint64_t)v, src);
  const uint64_t hi = __shfl_sync(0xffffffffu, (unsigned long long)(uint64_t)(v >> 64), src);
  return ((u128)hi << 64) | lo;
}

// Uniform draw as a 53-bit integer: U01 = draw_u53 * 2^-53 (same counter as draw_u01).
__device__ __forceinline__ uint64_t draw_u53(uint64_t seed, int64_t t, int s, int a) {
  const uint64_t ctr = 1ull + 128ull * (uint64_t)t + 2ull * (uint64_t)a + (uint64_t)s;
  return splitmix64_mix(seed + 0x9E3779B97F4A7C15ull * ctr) >> 11;
}

__device__ __forceinline__ uint64_t abs_bits(float v) { return (uint64_t)(fx_bits32(v) & 0x7FFFFFFFu); }
__device__ __forceinline__ uint64_t abs_bits(double v) { return fx_bits64(v) & ~(1ull << 63); }

// block-wide max of a 64-bit key (all threads call; result to all)
__device__ __forceinline__ uint64_t block_max_u64(uint64_t v, FxScratch& s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t u = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    v = u > v ? u : v;
  }
  if (lane == 0) s.key[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t m = 0;
    for (int w = 0; w < nw; ++w) m = s.key[w] > m ? s.key[w] : m;
    s.key[0] = m;
  }
  __syncthreads();
  const uint64_t r = s.key[0];
  __syncthreads();
  return r;
}

// Pass 1 of a selection: every warp's exact segment total into s.tot[warp]
// (segments of `seg` entries, lanes strided, loads issued four at a time).
template <typename WF>
__device__ __forceinline__ void fx_block_totals(const WF& wf, int64_t n, FxScratch& s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t seg = (n + nw - 1) / nw;
  seg = (seg + 31) / 32 * 32;
  const int64_t s0 = (int64_t)warp * seg;
  const int64_t s1 = min(n, s0 + seg);
  u128 acc = 0;
  int64_t p = s0 + lane;
  for (; p + 96 < s1; p += 128) {
    const u128 a0 = wf(p), a1 = wf(p + 32), a2 = wf(p + 64), a3 = wf(p + 96);
    acc += (a0 + a1) + (a2 + a3);
  }
  for (; p < s1; p += 32) acc += wf(p);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += shfl_xor_u128(acc, o);
  if (lane == 0) s.tot[warp] = acc;
  __syncthreads();
}

// Pass 2, after fx_block_totals over the same weights: thread 0 scans the
// segment totals and finds the warp whose segment holds the target (sel 1:
// floor(U T / 2^53); sel 2: the exact target tg_in; sel 0: none); that warp
// splits its segment into 32 contiguous runs, sums them, scans the run sums,
// and walks the run holding the target 32 entries at a time (a warp scan per
// chunk instead of one lane's chain of dependent loads).  Returns the index
// (-1 if none) and the exact total in *T_out.
template <typename WF>
__device__ int64_t fx_block_pick(const WF& wf, int64_t n, int sel, uint64_t U, u128 tg_in, u128* T_out,
                                 FxScratch& s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t seg = (n + nw - 1) / nw;
  seg = (seg + 31) / 32 * 32;
  const int64_t s0 = (int64_t)warp * seg;
  const int64_t s1 = min(n, s0 + seg);
  if (threadIdx.x == 0) {
    u128 run = 0;
    for (int w = 0; w < nw; ++w) {
      s.base[w] = run;
      run += s.tot[w];
    }
    s.T = run;
    s.found = -1;
    s.wstar = -1;
    if (sel != 0 && run > 0 && (sel == 1 || tg_in < run)) {
      const u128 tg = sel == 1 ? fx_target(U, run) : tg_in;
      s.target = tg;
      for (int w = 0; w < nw; ++w)
        if (s.tot[w] > 0 && s.base[w] + s.tot[w] > tg) { s.wstar = w; break; }
    }
  }
  __syncthreads();
  *T_out = s.T;
  if (warp == s.wstar) {
    const u128 tg = s.target;
    const int64_t len = s1 - s0;
    const int64_t run_len = (len + 31) / 32;
    const int64_t r0 = min(s1, s0 + (int64_t)lane * run_len);
    const int64_t r1 = min(s1, r0 + run_len);
    u128 mine = 0;
    {
      int64_t p = r0;
      for (; p + 7 < r1; p += 8) {
        const u128 a0 = wf(p), a1 = wf(p + 1), a2 = wf(p + 2), a3 = wf(p + 3);
        const u128 a4 = wf(p + 4), a5 = wf(p + 5), a6 = wf(p + 6), a7 = wf(p + 7);
        mine += ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
      }
      for (; p < r1; ++p) mine += wf(p);
    }
    // exclusive scan of the run sums over the lanes
    u128 incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u128 u = shfl_up_u128(incl, o);
      if (lane >= o) incl += u;
    }
    const u128 before = s.base[warp] + (incl - mine);
    const unsigned bal = __ballot_sync(0xffffffffu, mine > 0 && before + mine > tg);
    if (bal) {
      // the whole warp walks the run holding the target, 32 entries at a time
      const int src = __ffs(bal) - 1;
      u128 run = shfl_idx_u128(before, src);
      const int64_t q0 = __shfl_sync(0xffffffffu, (long long)r0, src);
      const int64_t q1 = __shfl_sync(0xffffffffu, (long long)r1, src);
      int64_t f = q1 - 1;
      for (int64_t c = q0; c < q1; c += 32) {
        const int64_t p = c + lane;
        const u128 v = p < q1 ? wf(p) : (u128)0;
        u128 pre = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const u128 u = shfl_up_u128(pre, o);
          if (lane >= o) pre += u;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, p < q1 && run + pre > tg);
        if (hit) {
          f = c + __ffs(hit) - 1;
          break;
        }
        run += shfl_idx_u128(pre, 31);
      }
      if (lane == 0) s.found = f;
    }
  }
  __syncthreads();
  const int64_t r = s.found;
  __syncthreads();
  return r;
}

// Exact draw over n weights wf(p) (u128): sel 0 forms the total only, 1
// draws with the uniform U, 2 selects with the exact target tg_in.  Returns
// the smallest p whose prefix sum exceeds the target (-1 when the total is
// zero or nothing is selected); *T_out receives the exact total.  All sums
// are exact integers, so the result does not depend on how the work is split.
template <typename WF>
__device__ int64_t fx_block_select(const WF& wf, int64_t n, int sel, uint64_t U, u128 tg_in, u128* T_out,
                                   FxScratch& s) {
  fx_block_totals(wf, n, s);
  return fx_block_pick(wf, n, sel, U, tg_in, T_out, s);
}

template <typename WF>
__device__ __forceinline__ int64_t fx_block_draw(const WF& wf, int64_t n, uint64_t U, bool draw, u128* T_out,
                                                 FxScratch& s) {
  return fx_block_select(wf, n, draw ? 1 : 0, U, (u128)0, T_out, s);
}

// Arg-max of keys kf(p) (u128 or uint64_t, compared as unsigned), ties to
// the smallest index; -1 when n == 0.
template <typename KF>
__device__ int64_t fx_block_argmax(const KF& kf, int64_t n, FxScratch& s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  u128 best = 0;
  int64_t bi = -1;
  for (int64_t p = threadIdx.x; p < n; p += blockDim.x) {
    const u128 v = (u128)kf(p);
    if (bi < 0 || v > best) { best = v; bi = p; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const u128 ov = shfl_xor_u128(best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, (long long)bi, o);
    if (oi >= 0 && (bi < 0 || ov > best || (ov == best && oi < bi))) { best = ov; bi = oi; }
  }
  if (lane == 0) { s.tot[warp] = best; s.idx[warp] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    u128 bv = 0;
    int64_t b = -1;
    for (int w = 0; w < nw; ++w) {
      const int64_t oi = s.idx[w];
      if (oi >= 0 && (b < 0 || s.tot[w] > bv || (s.tot[w] == bv && oi < b))) { bv = s.tot[w]; b = oi; }
    }
    s.found = b;
  }
  __syncthreads();
  const int64_t r = s.found;
  __syncthreads();
  return r;
}

// Largest bit pattern of n non-negative FP64 values (the largest value), per
// thread; loads issued four at a time.
__device__ __forceinline__ uint64_t max_bits_f64(const double* w, int64_t n) {
  uint64_t mb = 0;
  int64_t p = threadIdx.x;
  const int64_t st = blockDim.x;
  for (; p + 3 * st < n; p += 4 * st) {
    const uint64_t b0 = fx_bits64(w[p]), b1 = fx_bits64(w[p + st]), b2 = fx_bits64(w[p + 2 * st]),
                   b3 = fx_bits64(w[p + 3 * st]);
    const uint64_t m01 = b0 > b1 ? b0 : b1, m23 = b2 > b3 ? b2 : b3;
    const uint64_t m = m01 > m23 ? m01 : m23;
    mb = m > mb ? m : mb;
  }
  for (; p < n; p += st) {
    const uint64_t b = fx_bits64(w[p]);
    mb = b > mb ? b : mb;
  }
  return mb;
}

// Exact total of n non-negative FP64 values, rounded once to FP64.
__device__ __forceinline__ double fx_total_f64(const double* w, int64_t n, FxScratch& s) {
  uint64_t mb = max_bits_f64(w, n);
  mb = block_max_u64(mb, s);
  const int E = fx_scale_f64(mb, n);
  u128 T;
  (void)fx_block_draw([w, E](int64_t p) -> u128 { return fx_f64(w[p], E); }, n, 0, false, &T, s);
  return fx_to_double(T, E);
}

// Squared magnitude of an entry in fixed point (exact square, truncated once
// per component).
__device__ __forceinline__ u128 fx_abs2(float v, int E) { return fx_sq(v, E); }
__device__ __forceinline__ u128 fx_abs2(double v, int E) { return fx_sq(v, E); }
__device__ __forceinline__ u128 fx_abs2(cf32 v, int E) { return fx_sq(v.re, E) + fx_sq(v.im, E); }
__device__ __forceinline__ u128 fx_abs2(cf64 v, int E) { return fx_sq(v.re, E) + fx_sq(v.im, E); }

__device__ __forceinline__ uint64_t entry_max_bits(float v) { return abs_bits(v); }
__device__ __forceinline__ uint64_t entry_max_bits(double v) { return abs_bits(v); }
__device__ __forceinline__ uint64_t entry_max_bits(cf32 v) {
  const uint64_t a = abs_bits(v.re), b = abs_bits(v.im);
  return a > b ? a : b;
}
__device__ __forceinline__ uint64_t entry_max_bits(cf64 v) {
  const uint64_t a = abs_bits(v.re), b = abs_bits(v.im);
  return a > b ? a : b;
}

template <typename T> __device__ __forceinline__ int fx_entry_scale(uint64_t maxb, int64_t count);
template <> __device__ __forceinline__ int fx_entry_scale<float>(uint64_t mb, int64_t c) { return fx_scale_sq32((uint32_t)mb, c, 1); }
template <> __device__ __forceinline__ int fx_entry_scale<cf32>(uint64_t mb, int64_t c) { return fx_scale_sq32((uint32_t)mb, c, 2); }
template <> __device__ __forceinline__ int fx_entry_scale<double>(uint64_t mb, int64_t c) { return fx_scale_sq64(mb, c, 1); }
template <> __device__ __forceinline__ int fx_entry_scale<cf64>(uint64_t mb, int64_t c) { return fx_scale_sq64(mb, c, 2); }

}  // namespace rplu
