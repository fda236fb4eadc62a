// Device-side building blocks shared by the RPLU kernels: scalar traits for
// the four data types, the counter-based uniform draw, and block-wide FP64
// reductions, scans and arg-selections used by the two-stage sampler.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rplu.h"

namespace rplu {

constexpr int kMaxAttempts = 64;  // redraws of a row whose masked weights sum to 0

// Default write-back interval of the dense pass (steps between writes of the
// residual S; every interval gives the same results), the fastest measured
// on GB300: FP32 6 (32768^2, k = 256: 217.5 ms a call against 219.3 at 8 and
// 221.3 at 5), complex64 4 (16384^2, k = 128: 88.0 ms against 94.3 at 8 and
// 89.2 at 2), FP64 and complex128 1 (their updates are FP64-pipe bound).
inline int32_t default_pass_block(int32_t dtype) {
  return dtype == RPLU_F32 ? 6 : dtype == RPLU_C64 ? 4 : 1;
}

// Per-job device state of one factorization (lives in the workspace).
struct JobState {
  int64_t t;          // next step to draw
  int64_t cur;        // step being applied by the kernels that follow the draw
  int64_t k_done;     // steps completed (valid once done != 0)
  int64_t i, j;       // pivot of the current step
  double a_re, a_im;  // pivot value S(i, j) in FP64
  double T0;          // ||A||_F^2 (sum of the initial d)
  double unorm2;      // ||U(cur,:)||^2 (matrix-free form)
  int32_t done;       // 1: no further steps
  int32_t err;        // error bits (kErr*)
  int32_t attempt;    // redraw attempt of the current step (matrix-free form)
  int32_t redraw;     // matrix-free form: the row drawn at `cur` had zero masked weight
  int32_t skip;       // matrix-free form: the rest of this step's kernels do nothing
  int32_t fallback;   // bound-based draw: every proposal of step t was rejected, the
                      // exact-norm draw of the step is pending
};

enum : int32_t {
  kErrNonFinite = 1,   // non-finite entry / row norm in the input
  kErrZeroPivot = 2,   // forced pivot with value 0
  kErrBadGiven = 4,    // forced pivot out of range or repeated
  kErrTimeout = 8,     // a bounded device wait expired
  kErrInternal = 16,   // a kernel specialised for a step ran at another step
  kErrCancelled = 32,  // the caller cancelled the job (serving)
};

// Status of a finished job from its device-side state: the error bits in a
// fixed order of precedence, then the tolerance test (T_final > rel_tol^2 T0
// after all k steps).  *why receives a static string naming the reason.
inline rplu_status job_status(const JobState& st, double rel_tol, int64_t k, double T_final, const char** why) {
  *why = "";
  if (st.err & kErrNonFinite) { *why = "input has a non-finite entry (or x_i == y_j)"; return RPLU_ERR_INVALID; }
  if (st.err & kErrBadGiven) { *why = "forced pivot out of range or repeated"; return RPLU_ERR_INVALID; }
  if (st.err & kErrZeroPivot) { *why = "forced pivot has value zero"; return RPLU_ERR_INVALID; }
  if (st.err & kErrTimeout) { *why = "a bounded device wait expired"; return RPLU_ERR_TIMEOUT; }
  if (st.err & kErrInternal) { *why = "internal error: step bookkeeping mismatch"; return RPLU_ERR_CUDA; }
  if (rel_tol > 0.0 && st.k_done == k && k > 0 && T_final > rel_tol * rel_tol * st.T0) {
    *why = "rel_tol not reached within k steps";
    return RPLU_NOT_CONVERGED;
  }
  return RPLU_OK;
}

// ------------------------------------------------------------------ scalars

struct cf32 { float re, im; };
struct cf64 { double re, im; };

template <typename T> struct Traits;
template <> struct Traits<float> {
  using real = float;
  static constexpr bool kComplex = false;
  static constexpr int kVec = 4;  // elements per 16-byte vector
};
template <> struct Traits<double> {
  using real = double;
  static constexpr bool kComplex = false;
  static constexpr int kVec = 2;
};
template <> struct Traits<cf32> {
  using real = float;
  static constexpr bool kComplex = true;
  static constexpr int kVec = 2;
};
template <> struct Traits<cf64> {
  using real = double;
  static constexpr bool kComplex = true;
  static constexpr int kVec = 1;
};

__device__ __forceinline__ double abs2_d(float v) { return (double)v * (double)v; }
__device__ __forceinline__ double abs2_d(double v) { return v * v; }
__device__ __forceinline__ double abs2_d(cf32 v) { return (double)v.re * (double)v.re + (double)v.im * (double)v.im; }
__device__ __forceinline__ double abs2_d(cf64 v) { return v.re * v.re + v.im * v.im; }

__device__ __forceinline__ bool finite_v(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_v(double v) { return isfinite(v); }
__device__ __forceinline__ bool finite_v(cf32 v) { return isfinite(v.re) && isfinite(v.im); }
__device__ __forceinline__ bool finite_v(cf64 v) { return isfinite(v.re) && isfinite(v.im); }

template <typename T> __device__ __forceinline__ T zero_v() { return T{}; }
template <typename T> __device__ __forceinline__ T one_v();
template <> __device__ __forceinline__ float one_v<float>() { return 1.f; }
template <> __device__ __forceinline__ double one_v<double>() { return 1.0; }
template <> __device__ __forceinline__ cf32 one_v<cf32>() { return cf32{1.f, 0.f}; }
template <> __device__ __forceinline__ cf64 one_v<cf64>() { return cf64{1.0, 0.0}; }

__device__ __forceinline__ void to_d(float v, double& re, double& im) { re = v; im = 0.0; }
__device__ __forceinline__ void to_d(double v, double& re, double& im) { re = v; im = 0.0; }
__device__ __forceinline__ void to_d(cf32 v, double& re, double& im) { re = v.re; im = v.im; }
__device__ __forceinline__ void to_d(cf64 v, double& re, double& im) { re = v.re; im = v.im; }

template <typename T> __device__ __forceinline__ T from_d(double re, double im);
template <> __device__ __forceinline__ float from_d<float>(double re, double) { return (float)re; }
template <> __device__ __forceinline__ double from_d<double>(double re, double) { return re; }
template <> __device__ __forceinline__ cf32 from_d<cf32>(double re, double im) { return cf32{(float)re, (float)im}; }
template <> __device__ __forceinline__ cf64 from_d<cf64>(double re, double im) { return cf64{re, im}; }

// s - l * r, with fused multiply-adds in the working precision
__device__ __forceinline__ float fms(float s, float l, float r) { return fmaf(-l, r, s); }
__device__ __forceinline__ double fms(double s, double l, double r) { return fma(-l, r, s); }
__device__ __forceinline__ cf32 fms(cf32 s, cf32 l, cf32 r) {
  cf32 o;
  o.re = fmaf(l.im, r.im, fmaf(-l.re, r.re, s.re));
  o.im = fmaf(-l.im, r.re, fmaf(-l.re, r.im, s.im));
  return o;
}
__device__ __forceinline__ cf64 fms(cf64 s, cf64 l, cf64 r) {
  cf64 o;
  o.re = fma(l.im, r.im, fma(-l.re, r.re, s.re));
  o.im = fma(-l.im, r.re, fma(-l.re, r.im, s.im));
  return o;
}

// (nr + i ni) / (ar + i ai) in FP64 with true division: multiply by the
// conjugate, then divide both parts by |a|^2.
__device__ __forceinline__ void cdiv_d(double nr, double ni, double ar, double ai, double& qr, double& qi) {
  if (ai == 0.0) {
    qr = nr / ar;
    qi = ni / ar;
    return;
  }
  double den = ar * ar + ai * ai;
  qr = (nr * ar + ni * ai) / den;
  qi = (ni * ar - nr * ai) / den;
}

// ------------------------------------------------------------------ draws

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform in [0, 1) for step t, stage s (0 row, 1 column), redraw attempt a:
// output number 1 + 128 t + 2 a + s of the SplitMix64 stream seeded with seed.
__device__ __forceinline__ double draw_u01(uint64_t seed, int64_t t, int s, int a) {
  const uint64_t ctr = 1ull + 128ull * (uint64_t)t + 2ull * (uint64_t)a + (uint64_t)s;
  const uint64_t z = splitmix64_mix(seed + 0x9E3779B97F4A7C15ull * ctr);
  return (double)(z >> 11) * 0x1.0p-53;
}

// ------------------------------------------------------ block collectives
// All helpers assume blockDim.x is a multiple of 32 and at most 1024, and are
// called by every thread of the block.

__device__ __forceinline__ double warp_incl_scan(double v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive prefix over threads in thread order; returns this thread's
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ double block_excl_scan(double v, double* total, double* sh /* >= 33 doubles */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double incl = warp_incl_scan(v);
  double wex = __shfl_up_sync(0xffffffffu, incl, 1);  // in-warp exclusive prefix
  if (lane == 0) wex = 0.0;
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const double w = lane < nw ? sh[lane] : 0.0;
    const double wi = warp_incl_scan(w);
    double we = __shfl_up_sync(0xffffffffu, wi, 1);  // exclusive prefix of warp totals
    if (lane == 0) we = 0.0;
    sh[lane] = we;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  const double excl = (warp == 0) ? wex : sh[warp] + wex;
  *total = sh[32];
  __syncthreads();
  return excl;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  double tot;
  (void)block_excl_scan(v, &tot, sh);
  return tot;
}

__device__ __forceinline__ int64_t block_min_i64(int64_t v, int64_t* sh /* >= 32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    int64_t u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u < v ? u : v;
  }
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < nw ? sh[lane] : INT64_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      int64_t u = __shfl_xor_sync(0xffffffffu, w, o);
      w = u < w ? u : w;
    }
    if (lane == 0) sh[0] = w;
  }
  __syncthreads();
  int64_t r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int64_t block_max_i64(int64_t v, int64_t* sh) {
  return -block_min_i64(-v, sh);
}

// (value, index) argmax; ties to the smallest index.  Index -1 = no candidate.
__device__ __forceinline__ bool better(double v, int64_t i, double bv, int64_t bi) {
  if (i < 0) return false;
  if (bi < 0) return true;
  return v > bv || (v == bv && i < bi);
}

__device__ __forceinline__ void block_argmax(double& v, int64_t& i, double* shv, int64_t* shi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double uv = __shfl_xor_sync(0xffffffffu, v, o);
    int64_t ui = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(uv, ui, v, i)) { v = uv; i = ui; }
  }
  if (lane == 0) { shv[warp] = v; shi[warp] = i; }
  __syncthreads();
  if (warp == 0) {
    double wv = lane < nw ? shv[lane] : -1.0;
    int64_t wi = lane < nw ? shi[lane] : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double uv = __shfl_xor_sync(0xffffffffu, wv, o);
      int64_t ui = __shfl_xor_sync(0xffffffffu, wi, o);
      if (better(uv, ui, wv, wi)) { wv = uv; wi = ui; }
    }
    if (lane == 0) { shv[0] = wv; shi[0] = wi; }
  }
  __syncthreads();
  v = shv[0];
  i = shi[0];
  __syncthreads();
}

// Shared scratch of the block collectives above.
struct BlockScratch {
  double dv[40];
  int64_t iv[40];
};

}  // namespace rplu
