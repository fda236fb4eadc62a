// Grid-wide exact inverse-CDF draw over a long weight vector (n up to 10^8 and
// more): the weights are split into chunks, one CTA per chunk, in two passes
// (the largest weight's bit pattern, for the fixed-point scale; then each
// chunk's exact fixed-point total), and one CTA then scans the chunk totals,
// forms the target floor(U T / 2^53) from the exact total T, and selects
// within the chunk that holds it (sampler.cuh with the exact target).  Integer
// sums do not depend on how the work is split, so the drawn index is the
// single-CTA draw's bit for bit: the smallest p whose prefix sum exceeds the
// target.  The one-CTA draw reads the vector three times from one SM; this
// reads it twice from all of them.
#pragma once

#include "kernels.h"
#include "sampler.cuh"

namespace rplu {

constexpr int kGdThreads = 256;  // threads of the per-chunk passes (chunk shape: grid_draw_shape)

// The workspace of one draw stage is a GridDraw (kernels.h): the running
// maximum of the keys, reset to 0 by the select kernel that reads it, and the
// chunks' exact totals (u128 each).
__device__ __forceinline__ u128* gd_parts(const GridDraw& g) { return (u128*)g.part; }

// Pass 1 (one CTA per chunk, all threads): the chunk's largest key into g.maxb.
template <typename KF>
__device__ __forceinline__ void gd_max(const KF& kf, int64_t n, const GridDraw& g, FxScratch& s) {
  const int64_t c0 = (int64_t)blockIdx.x * g.len;
  const int64_t c1 = min(n, c0 + g.len);
  uint64_t m = 0;
  for (int64_t p = c0 + threadIdx.x; p < c1; p += blockDim.x) {
    const uint64_t k = kf(p);
    m = k > m ? k : m;
  }
  m = block_max_u64(m, s);
  if (threadIdx.x == 0 && m) atomicMax(g.maxb, (unsigned long long)m);
}

// Pass 2 (one CTA per chunk, all threads): the chunk's exact total into g.part.
template <typename WF>
__device__ __forceinline__ void gd_part(const WF& wf, int64_t n, const GridDraw& g, FxScratch& s) {
  const int64_t c0 = (int64_t)blockIdx.x * g.len;
  const int64_t c1 = min(n, c0 + g.len);
  const int64_t len = c1 > c0 ? c1 - c0 : 0;
  auto wl = [&wf, c0](int64_t p) -> u128 { return wf(c0 + p); };
  fx_block_totals(wl, len, s);
  if (threadIdx.x == 0) {
    u128 tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s.tot[w];
    gd_parts(g)[blockIdx.x] = tot;
  }
}

// Select (one CTA, all threads, after both passes over the same weights): the
// exact total into *T_out; with draw, the smallest index whose prefix sum
// exceeds floor(U T / 2^53) (-1 when the total is 0).
template <typename WF>
__device__ int64_t gd_select(const WF& wf, int64_t n, const GridDraw& g, bool draw, uint64_t U, u128* T_out,
                             FxScratch& s) {
  __shared__ u128 sh_T, sh_tgl;
  __shared__ long long sh_c;
  if (threadIdx.x == 0) {
    u128 T = 0;
    for (int64_t c = 0; c < g.chunks; ++c) T += gd_parts(g)[c];
    long long cstar = -1;
    u128 tgl = 0;
    if (draw && T > 0) {
      const u128 tg = fx_target(U, T);
      u128 b = 0;
      for (int64_t c = 0; c < g.chunks; ++c) {
        const u128 pc = gd_parts(g)[c];
        if (pc > 0 && b + pc > tg) {
          cstar = c;
          tgl = tg - b;
          break;
        }
        b += pc;
      }
    }
    sh_T = T;
    sh_tgl = tgl;
    sh_c = cstar;
  }
  __syncthreads();
  *T_out = sh_T;
  const long long cstar = sh_c;
  const u128 tgl = sh_tgl;
  __syncthreads();
  if (cstar < 0) return -1;
  const int64_t c0 = (int64_t)cstar * g.len;
  const int64_t c1 = min(n, c0 + g.len);
  auto wl = [&wf, c0](int64_t p) -> u128 { return wf(c0 + p); };
  u128 Tl;
  const int64_t li = fx_block_select(wl, c1 - c0, 2, 0, tgl, &Tl, s);
  return li < 0 ? -1 : c0 + li;
}

}  // namespace rplu
