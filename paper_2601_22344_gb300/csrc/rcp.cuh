// Reciprocals built on the hardware approximations (FP32 for generated
// Cauchy entries, FP64 for the near-field terms of the row-norm bounds).
//
// rcp_nr: one Newton-Raphson correction of the hardware approximation y0
// (faithful: within one ulp of 1/b), with the residual 1 - b*y0 formed exactly
// by one fused multiply-add and the correction y0 + y0*e applied by one FMA in
// round-to-nearest: Markstein's FMA correction step (Markstein, "Computation
// of elementary functions on the IBM RISC System/6000 processor", IBM J. Res.
// Dev. 34(1), 1990; Muller et al., Handbook of Floating-Point Arithmetic,
// ch. 4).  No branches.  For 2^-124 <= |b| < 2^124 (operand and reciprocal
// normal; see rcp_nr_range) the result is the correctly rounded reciprocal:
// tests/test_gpu_rcp.py checks every such operand (all significands, both
// signs, every exponent) bit for bit against __frcp_rn.
#pragma once

namespace rplu {

__device__ __forceinline__ float rcp_nr(float b) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(b));
  const float e = __fmaf_rn(-b, y, 1.0f);
  return __fmaf_rn(y, e, y);
}

// True when v = 1/b (correctly rounded) certifies 2^-124 <= |b| < 2^124, the
// range where rcp_nr is exact: |v| within [2^-123, 2^123].
__device__ __forceinline__ bool rcp_nr_range(float v) {
  const float a = fabsf(v);
  return a >= 0x1p-123f && a <= 0x1p123f;
}

// FP64 reciprocal for the exact near-field terms of the row-norm bounds: the
// hardware approximation (rcp.approx.ftz.f64) refined by two Newton-Raphson
// steps, each in Markstein's FMA form (residual e = 1 - b*y by one fused
// multiply-add, then y + y*e); the relative error squares at every step.
// For normal b with a normal reciprocal the result is within one ulp of 1/b
// (tests/test_gpu_rcp.py compares it with 1.0/b on operands spread over the
// exponent range).  Cheaper on the FP64 pipe than IEEE division.
__device__ __forceinline__ double rcp_nr64(double b) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(b));
  double e = fma(-b, y, 1.0);
  y = fma(y, e, y);
  e = fma(-b, y, 1.0);
  return fma(y, e, y);
}

}  // namespace rplu
