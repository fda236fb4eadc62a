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
#include "cluster.cuh"
#include "sampler.cuh"
#include "tma.cuh"

namespace rplu {
namespace {

constexpr int kClMaxBlk = 8;

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
