// Packed FP32 pairs (sm_100+ f32x2 instructions, through the compiler's
// builtins so that it schedules them like any other instruction): one
// instruction applies the same operation to two lanes; each lane is rounded
// exactly like the scalar instruction (a - b = a + (-b) exactly).  Used to halve the FP32 issue cost of the generated
// Cauchy kernels, two matrix rows per pair.
#pragma once

namespace rplu {

__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 f2_splat(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }

}  // namespace rplu
