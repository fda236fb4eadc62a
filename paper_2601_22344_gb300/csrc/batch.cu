// rplu_batch: many independent small factorizations (hierarchical-matrix
// blocks, paper Sec. 5.1).  First version: each job runs the dense-form
// kernels in turn on the caller's stream; Cauchy jobs are materialised on the
// device first.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "rplu.h"

namespace rplu {
namespace {

template <typename T>
__global__ void k_materialise_cauchy(const T* x, const T* y, int64_t n, int64_t m, T* A) {
  const int64_t total = n * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / m, q = e - p * m;
    A[e] = (T)1 / (x[p] - y[q]);
  }
}

}  // namespace
}  // namespace rplu

using namespace rplu;

extern "C" rplu_status rplu_batch(rplu_job* jobs, int32_t njobs, const rplu_opts* opts) {
  rplu_opts o;
  if (opts) o = *opts;
  else rplu_opts_init(&o);
  if (njobs < 0 || (njobs > 0 && !jobs)) return RPLU_ERR_INVALID;
  if (o.pivot != RPLU_PIVOT_RANDOM && o.pivot != RPLU_PIVOT_C2) return RPLU_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)o.stream;
  rplu_status worst = RPLU_OK;
  for (int32_t b = 0; b < njobs; ++b) {
    rplu_job& jb = jobs[b];
    jb.k_done = 0;
    jb.rel_res = NAN;
    rplu_status st = RPLU_OK;
    if (jb.dtype != RPLU_F32 && jb.dtype != RPLU_F64) st = RPLU_ERR_INVALID;
    if (jb.kind != 0 && jb.kind != 1) st = RPLU_ERR_INVALID;
    if (st == RPLU_OK && (jb.n < 0 || jb.m < 0 || jb.k_max < 0 || jb.k_max > (jb.n < jb.m ? jb.n : jb.m)))
      st = RPLU_ERR_INVALID;
    void* A = nullptr;
    const int64_t w = jb.dtype == RPLU_F32 ? 4 : 8;
    if (st == RPLU_OK && jb.kind == 1) {
      cudaPointerAttributes at;
      bool dev = cudaPointerGetAttributes(&at, jb.x) == cudaSuccess &&
                 (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
      (void)cudaGetLastError();
      const void* xd = jb.x;
      const void* yd = jb.y;
      void* xs = nullptr;
      void* ys = nullptr;
      if (cudaMallocAsync(&A, (size_t)(jb.n * jb.m * w + 16), s) != cudaSuccess) st = RPLU_ERR_NOMEM;
      if (st == RPLU_OK && !dev) {
        cudaMallocAsync(&xs, (size_t)(jb.n * w + 16), s);
        cudaMallocAsync(&ys, (size_t)(jb.m * w + 16), s);
        cudaMemcpyAsync(xs, jb.x, jb.n * w, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(ys, jb.y, jb.m * w, cudaMemcpyHostToDevice, s);
        xd = xs;
        yd = ys;
      }
      if (st == RPLU_OK && jb.n * jb.m > 0) {
        const int64_t blocks = (jb.n * jb.m + 255) / 256;
        const unsigned g = (unsigned)(blocks > 4096 ? 4096 : blocks);
        if (jb.dtype == RPLU_F32)
          k_materialise_cauchy<float><<<g, 256, 0, s>>>((const float*)xd, (const float*)yd, jb.n, jb.m, (float*)A);
        else
          k_materialise_cauchy<double><<<g, 256, 0, s>>>((const double*)xd, (const double*)yd, jb.n, jb.m, (double*)A);
      }
      if (xs) cudaFreeAsync(xs, s);
      if (ys) cudaFreeAsync(ys, s);
    }
    if (st == RPLU_OK) {
      rplu_opts jo = o;
      jo.dtype = jb.dtype;
      jo.rel_tol = jb.rel_tol;
      jo.lda = jb.kind == 1 ? jb.m : jb.lda;
      jo.overwrite_input = jb.kind == 1;
      std::vector<double> T(jb.k_max + 1, 0.0);
      jo.T_hist = T.data();
      int64_t kd = 0;
      st = rplu_dense(jb.kind == 1 ? A : jb.A, jb.n, jb.m, jb.k_max, jb.seed, &jo, jb.I, jb.J, jb.L, jb.U, &kd);
      jb.k_done = kd;
      if (st == RPLU_OK || st == RPLU_NOT_CONVERGED) jb.rel_res = T[0] > 0 ? std::sqrt(T[kd] / T[0]) : 0.0;
    }
    if (A) cudaFreeAsync(A, s);
    jb.status = st;
    if (st != RPLU_OK && (worst == RPLU_OK || worst == RPLU_NOT_CONVERGED)) worst = st;
  }
  cudaStreamSynchronize(s);
  return worst;
}
