// FP32 reciprocal for generated Cauchy entries.
//
// rcp_nr: Newton-Raphson from the hardware approximation, two steps, each
// residual 1 - b*y formed exactly by one fused multiply-add and the last
// correction applied with one FMA in round-to-nearest (Markstein, "Computation
// of elementary functions on the IBM RISC System/6000 processor", IBM J. Res.
// Dev. 34(1), 1990; Muller et al., Handbook of Floating-Point Arithmetic,
// ch. 4).  No branches.  Valid where the operand and its reciprocal are
// normal: 2^-124 <= |b| < 2^124 (see rcp_nr_range).  In that range it returns the
// correctly rounded reciprocal; tests/test_gpu_rcp.py checks it bit for bit
// against __frcp_rn for every significand, both signs and exponents across the
// range.
#pragma once

namespace rplu {

__device__ __forceinline__ float rcp_nr(float b) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(b));
  float e = __fmaf_rn(-b, y, 1.0f);
  y = __fmaf_rn(y, e, y);
  e = __fmaf_rn(-b, y, 1.0f);
  return __fmaf_rn(y, e, y);
}

// True when v = 1/b (correctly rounded) certifies 2^-124 <= |b| < 2^124, the
// range where rcp_nr is exact: |v| within [2^-123, 2^123].
__device__ __forceinline__ bool rcp_nr_range(float v) {
  const float a = fabsf(v);
  return a >= 0x1p-123f && a <= 0x1p123f;
}

}  // namespace rplu
