// Cluster-wide pieces of the exact inverse-CDF draw (sampler.cuh) for a
// thread-block cluster of kCl CTAs: each CTA owns a contiguous range of the
// weights, partial maxima and exact fixed-point sums are exchanged through
// distributed shared memory (mapa + st.shared::cluster) between hardware
// cluster barriers, and the CTA whose range holds the target selects the
// index and sends it to the others.  The sums are exact integers, so the
// selected index equals that of a single-CTA draw over the same weights.
#pragma once

#include "common.cuh"
#include "sampler.cuh"
#include "tma.cuh"

namespace rplu {
namespace {

constexpr int kCl = 8;
constexpr int kClThreads = 512;

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// hardware barrier over every thread of the cluster, release/acquire
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(cta));
  return r;
}
__device__ __forceinline__ void cl_st_u64(uint32_t addr, uint64_t v) {
  asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

// Loads through L2 only: values another CTA of the cluster wrote in this launch.
__device__ __forceinline__ float ld_l2(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_l2(const double* p) { return __ldcg(p); }
__device__ __forceinline__ cf32 ld_l2(const cf32* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cf32{v.x, v.y};
}
__device__ __forceinline__ cf64 ld_l2(const cf64* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return cf64{v.x, v.y};
}

// Exchange area, double buffered: exchange e uses buffer e & 1, so an
// exchange may start while another CTA still reads the previous one (a CTA
// that writes exchange e + 2 has passed the barrier of exchange e + 1, which
// every CTA reaches only after reading exchange e).
struct ClShared {
  uint64_t v0[2][kCl];  // per-CTA values of the exchange (max bits, or low words of sums)
  uint64_t v1[2][kCl];  // high words of sums
  int64_t idx[2];       // selected index, sent by the owner
};

// Thread 0 writes (a, b) into slot `rank` of buffer `buf` of every CTA's exchange area.
__device__ __forceinline__ void cl_send(ClShared& x, int buf, uint32_t rank, uint64_t a, uint64_t b) {
  if (threadIdx.x == 0)
    for (uint32_t c = 0; c < kCl; ++c) {
      cl_st_u64(cl_map(&x.v0[buf][rank], c), a);
      cl_st_u64(cl_map(&x.v1[buf][rank], c), b);
    }
}
__device__ __forceinline__ void cl_send_idx(ClShared& x, int buf, int64_t i) {
  if (threadIdx.x == 0)
    for (uint32_t c = 0; c < kCl; ++c) cl_st_u64(cl_map(&x.idx[buf], c), (uint64_t)i);
}

// Cluster-wide exact selection over the weights wf of this CTA's range
// [lo, lo + len): returns the global index (same in every CTA) or -1, and the
// exact total in *T.  Contains cluster barriers: every CTA calls it.
template <typename WF>
__device__ int64_t cl_draw(const WF& wf, int64_t lo, int64_t len, uint64_t U, u128* T, ClShared& x, FxScratch& sh,
                           uint32_t rank, int& ex) {
  u128 part;
  auto local = [&wf, lo](int64_t p) -> u128 { return wf(lo + p); };
  fx_block_totals(local, len, sh);  // per-warp totals stay in sh for the pick below
  (void)fx_block_pick(local, len, 0, 0, (u128)0, &part, sh);
  const int b0 = ex++ & 1;
  cl_send(x, b0, rank, (uint64_t)part, (uint64_t)(part >> 64));
  cl_sync();
  u128 tot = 0, base = 0;
  u128 sums[kCl];
#pragma unroll
  for (int c = 0; c < kCl; ++c) {
    sums[c] = ((u128)x.v1[b0][c] << 64) | x.v0[b0][c];
    tot += sums[c];
  }
  *T = tot;
  int owner = -1;
  u128 tg = 0;
  if (tot > 0) {
    tg = fx_target(U, tot);
    for (int c = 0; c < kCl; ++c) {
      if (sums[c] > 0 && base + sums[c] > tg) {
        owner = c;
        break;
      }
      base += sums[c];
    }
  }
  const int b1 = ex++ & 1;
  if ((int)rank == owner) {
    u128 dummy;
    const int64_t f = fx_block_pick(local, len, 2, 0, tg - base, &dummy, sh);
    cl_send_idx(x, b1, f >= 0 ? lo + f : -1);
  }
  cl_sync();
  return owner >= 0 ? x.idx[b1] : -1;
}

// Cluster-wide maximum of per-thread bit patterns.
__device__ __forceinline__ uint64_t cl_max(uint64_t mb, ClShared& x, FxScratch& sh, uint32_t rank, int& ex) {
  mb = block_max_u64(mb, sh);
  const int b = ex++ & 1;
  cl_send(x, b, rank, mb, 0);
  cl_sync();
  uint64_t g = 0;
#pragma unroll
  for (int c = 0; c < kCl; ++c) g = x.v0[b][c] > g ? x.v0[b][c] : g;
  return g;
}

// Cluster-wide exact total of the weights wf over this CTA's range [lo, lo + len).
template <typename WF>
__device__ u128 cl_total(const WF& wf, int64_t lo, int64_t len, ClShared& x, FxScratch& sh, uint32_t rank, int& ex) {
  u128 part;
  auto local = [&wf, lo](int64_t p) -> u128 { return wf(lo + p); };
  fx_block_totals(local, len, sh);
  (void)fx_block_pick(local, len, 0, 0, (u128)0, &part, sh);
  const int b = ex++ & 1;
  cl_send(x, b, rank, (uint64_t)part, (uint64_t)(part >> 64));
  cl_sync();
  u128 tot = 0;
#pragma unroll
  for (int c = 0; c < kCl; ++c) tot += ((u128)x.v1[b][c] << 64) | x.v0[b][c];
  return tot;
}

// Cluster-wide arg-max of the keys kf over this CTA's range [lo, lo + len):
// the largest key, ties to the smallest index; -1 and key 0 when every key
// is 0.  Contains cluster barriers: every CTA calls it.
template <typename KF>
__device__ int64_t cl_argmax(const KF& kf, int64_t lo, int64_t len, ClShared& x, FxScratch& sh, uint32_t rank,
                             int& ex, uint64_t* key_out) {
  auto local = [&kf, lo](int64_t p) -> uint64_t { return kf(lo + p); };
  const int64_t li = fx_block_argmax(local, len, sh);
  const uint64_t key = li >= 0 ? kf(lo + li) : 0ull;
  const int b = ex++ & 1;
  cl_send(x, b, rank, key, li >= 0 ? (uint64_t)(lo + li) : ~0ull);
  cl_sync();
  uint64_t bk = 0, bi = ~0ull;
#pragma unroll
  for (int c = 0; c < kCl; ++c) {
    const uint64_t kc = x.v0[b][c], ic = x.v1[b][c];
    if (ic != ~0ull && (kc > bk || (kc == bk && ic < bi))) {
      bk = kc;
      bi = ic;
    }
  }
  *key_out = bk;
  return (bk == 0 || bi == ~0ull) ? -1 : (int64_t)bi;
}

}  // namespace
}  // namespace rplu
