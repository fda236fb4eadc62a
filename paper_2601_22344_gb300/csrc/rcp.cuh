// FP32 reciprocal for generated Cauchy entries.
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

}  // namespace rplu
