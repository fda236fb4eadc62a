// Entries of Cauchy-like matrices generated from their generators (Eq.
// cauchy-like): working-precision scalar helpers shared by the exact-norm
// kernels (cauchy_like.cu) and the bound / rejection-sampling kernels
// (cauchy_bh.cu).
#pragma once

#include "common.cuh"

namespace rplu {

__device__ __forceinline__ float rcp_fast(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ double rcp_fast(double v) { return 1.0 / v; }

__device__ __forceinline__ float re_of(float v) { return v; }
__device__ __forceinline__ double re_of(double v) { return v; }
__device__ __forceinline__ float re_of(cf32 v) { return v.re; }
__device__ __forceinline__ double re_of(cf64 v) { return v.re; }
__device__ __forceinline__ float im_of(float) { return 0.f; }
__device__ __forceinline__ double im_of(double) { return 0.0; }
__device__ __forceinline__ float im_of(cf32 v) { return v.im; }
__device__ __forceinline__ double im_of(cf64 v) { return v.im; }

// a * b in the working precision (complex: plain product)
__device__ __forceinline__ float mul_v(float a, float b) { return a * b; }
__device__ __forceinline__ double mul_v(double a, double b) { return a * b; }
__device__ __forceinline__ cf32 mul_v(cf32 a, cf32 b) {
  return cf32{fmaf(a.re, b.re, -a.im * b.im), fmaf(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ cf64 mul_v(cf64 a, cf64 b) {
  return cf64{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ float add_v(float a, float b) { return a + b; }
__device__ __forceinline__ double add_v(double a, double b) { return a + b; }
__device__ __forceinline__ cf32 add_v(cf32 a, cf32 b) { return cf32{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cf64 add_v(cf64 a, cf64 b) { return cf64{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ float sub_v(float a, float b) { return a - b; }
__device__ __forceinline__ double sub_v(double a, double b) { return a - b; }
__device__ __forceinline__ cf32 sub_v(cf32 a, cf32 b) { return cf32{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cf64 sub_v(cf64 a, cf64 b) { return cf64{a.re - b.re, a.im - b.im}; }

// s / z in the working precision: FP64 data with FP64 division; FP32 data
// in FP32 (real: correctly rounded division; complex: s conj(z) times the
// correctly rounded reciprocal of |z|^2), off the FP64 pipe.
__device__ __forceinline__ float div_v(float s, float z) { return __fdiv_rn(s, z); }
__device__ __forceinline__ double div_v(double s, double z) { return s / z; }
__device__ __forceinline__ cf32 div_v(cf32 s, cf32 z) {
  const float inv = __frcp_rn(fmaf(z.re, z.re, z.im * z.im));
  return cf32{fmaf(s.re, z.re, s.im * z.im) * inv, fmaf(s.im, z.re, -s.re * z.im) * inv};
}
__device__ __forceinline__ cf64 div_v(cf64 s, cf64 z) {
  double qr, qi;
  cdiv_d(s.re, s.im, z.re, z.im, qr, qi);
  return cf64{qr, qi};
}

// Entry of the generated residual: (sum_l g_l b_l) / (x - y).
template <typename T, int P>
__device__ __forceinline__ T entry_gen(const T (&g)[P], const T (&b)[P], T x, T y) {
  T s = mul_v(g[0], b[0]);
#pragma unroll
  for (int l = 1; l < P; ++l) s = add_v(s, mul_v(g[l], b[l]));
  return div_v(s, sub_v(x, y));
}

}  // namespace rplu
