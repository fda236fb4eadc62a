// The dense form's two-stage pivot draw (Sec. 4.1) on a cluster of 8 CTAs.
//
// CTA c of the cluster owns rows [c*RS, (c+1)*RS) of d and columns
// [c*CS, (c+1)*CS) of the pivot row.  Each stage: every CTA forms the maximum
// of its weights' bit patterns and its exact fixed-point partial sum; the
// partial results are exchanged through distributed shared memory (mapa +
// st.shared::cluster) between hardware cluster barriers; every CTA then knows
// the total and the target, and the CTA whose range holds the target selects
// the index within it and sends it to the others.  The draws equal those of
// the single-CTA sampler (k_dense_sample) exactly: the sums are exact
// integers, so the split does not change the selected index.  Used for
// RPLU_PIVOT_RANDOM; the other modes keep the single-CTA kernel.
#include "common.cuh"
#include "kernels.h"
#include "sampler.cuh"
#include "tma.cuh"

namespace rplu {
namespace {

constexpr int kCl = 8;
constexpr int kClThreads = 512;
constexpr int kClMaxBlk = 8;

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

template <typename T>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClThreads) k_dense_sample_cl(DenseLaunch a) {
  __shared__ FxScratch sh;
  __shared__ ClShared x;
  __shared__ T Li[kClMaxBlk];
  JobState* st = a.st;
  if (st->done) return;  // same value in every CTA: nothing writes it before the final barrier
  const uint32_t rank = cl_rank();
  const int64_t t = st->t;
  const int r = (int)(t % a.blk);
  const int64_t t0 = t - r;
  const T* S = (const T*)a.S;
  const T* Lout = (const T*)a.L;
  double* d = a.d;
  const uint8_t* col_used = a.col_used;
  const int64_t RS = (a.n + kCl - 1) / kCl;
  const int64_t rlo = min(a.n, (int64_t)rank * RS), rlen = min(a.n, rlo + RS) - rlo;
  int64_t CS = (a.lds + kCl - 1) / kCl;
  CS = (CS + 3) / 4 * 4;
  const int64_t qlo = min(a.lds, (int64_t)rank * CS), qhi = min(a.lds, qlo + CS);
  const int64_t mlen = max((int64_t)0, min(a.m, qhi) - qlo);

  int ex = 0;  // exchanges so far (selects the buffer)
  const uint64_t gmb = cl_max(max_bits_f64(d + rlo, rlen), x, sh, rank, ex);
  const int Er = fx_scale_f64(gmb, a.n);
  // d is read through L2: a redraw zeroes an entry between two passes over it
  auto dw = [d, Er](int64_t p) -> u128 { return fx_f64(__ldcg(d + p), Er); };
  T* urow = (T*)a.U + t * a.m;
  T* ub = (T*)a.ublk;
  T* rh = ub + (int64_t)r * a.lds;
  int64_t i = -1, j = -1;
  bool ok = false;
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
    // S^(t)(i,:) on this CTA's columns: the stored row minus the pending updates
    if (threadIdx.x < r) Li[threadIdx.x] = Lout[(t0 + threadIdx.x) * a.n + i];
    __syncthreads();
    const T* srow = S + i * a.lds;
    uint64_t cb = 0;
    for (int64_t q = qlo + threadIdx.x; q < qhi; q += kClThreads) {
      T v = q < a.m ? srow[q] : zero_v<T>();
      for (int s = 0; s < r; ++s) v = fms(v, Li[s], ub[(int64_t)s * a.lds + q]);
      v = (q < a.m && !col_used[q]) ? v : zero_v<T>();
      rh[q] = v;
      if (q < a.m) urow[q] = v;
      const uint64_t b = entry_max_bits(v);
      cb = b > cb ? b : cb;
    }
    const uint64_t gcb = cl_max(cb, x, sh, rank, ex);  // its barrier also orders the row writes
    const int Ec = fx_entry_scale<T>(gcb, a.m);
    const T* rr = rh;
    auto cw = [rr, Ec](int64_t q) -> u128 { return fx_abs2(rr[q], Ec); };
    u128 Rfx;
    j = cl_draw(cw, qlo, mlen, draw_u53(a.seed, t, 1, attempt), &Rfx, x, sh, rank, ex);
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
    to_d(ld_l2(rh + j), ar, ai);  // written by the CTA that owns column j
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
  st->cur = t;
  st->t = t + 1;
}

}  // namespace

cudaError_t dense_sample_cluster(int32_t dtype, const DenseLaunch& a, cudaStream_t s) {
  switch (dtype) {
    case RPLU_F32: k_dense_sample_cl<float><<<kCl, kClThreads, 0, s>>>(a); break;
    case RPLU_F64: k_dense_sample_cl<double><<<kCl, kClThreads, 0, s>>>(a); break;
    case RPLU_C64: k_dense_sample_cl<cf32><<<kCl, kClThreads, 0, s>>>(a); break;
    case RPLU_C128: k_dense_sample_cl<cf64><<<kCl, kClThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rplu
