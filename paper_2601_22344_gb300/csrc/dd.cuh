// Double-double arithmetic for the CUR forms' core A(I,J)^{-1}: a value is an
// unevaluated sum hi + lo of two doubles with |lo| <= ulp(hi) / 2, about 106
// significant bits.  Built from error-free transformations: TwoSum (Knuth, The
// Art of Computer Programming vol. 2), TwoProduct with one FMA (the exact
// rounding error of a product), and the double-double sum and product of Hida,
// Li & Bailey ("Algorithms for quad-double precision floating point
// arithmetic", 2001).  Keeping the block-inverse update (Eq.
// block-inverse-update) in this precision makes its rounding, which grows like
// eps^2 cond(A(I,J))^2 here, smaller than the eps cond that the FP64 entries
// already carry, so the O(k^2) update becomes as accurate as a QR of A(I,J).
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#include <cuda_runtime.h>
#define RPLU_DD __host__ __device__ __forceinline__
#else
#define RPLU_DD inline  // host C++ (the CPU test of these functions)
#endif

namespace rplu {

struct dd {
  double hi, lo;
};

RPLU_DD dd dd_from(double a) { return dd{a, 0.0}; }

// s + e = a + b exactly
RPLU_DD dd two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  return dd{s, (a - (s - bb)) + (b - bb)};
}

// s + e = a + b exactly, given |a| >= |b|
RPLU_DD dd quick_two_sum(double a, double b) {
  const double s = a + b;
  return dd{s, b - (s - a)};
}

// p + e = a * b exactly (the FMA computes a * b - p without rounding the product)
RPLU_DD dd two_prod(double a, double b) {
  const double p = a * b;
  return dd{p, fma(a, b, -p)};
}

RPLU_DD dd dd_add(dd a, dd b) {
  const dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  dd r = quick_two_sum(s.hi, s.lo + t.hi);
  return quick_two_sum(r.hi, r.lo + t.lo);
}

RPLU_DD dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }

RPLU_DD dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo = fma(a.hi, b.lo, fma(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}

// a double times a double-double
RPLU_DD dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo = fma(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// 1 / a by one Newton correction of the FP64 quotient: q1 = 1 / a.hi, then
// q1 + q1 (1 - a q1), the residual 1 - a q1 formed in double-double
RPLU_DD dd dd_recip(dd a) {
  const double q1 = 1.0 / a.hi;
  const dd r = dd_add(dd_from(1.0), dd_neg(dd_mul_d(a, q1)));
  return quick_two_sum(q1, q1 * r.hi);
}

#if defined(__CUDACC__)
// butterfly sum of a warp's double-double values (fixed order)
__device__ __forceinline__ dd dd_warp_sum(dd v) {
  for (int o = 16; o > 0; o >>= 1) {
    const dd w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = dd_add(v, w);
  }
  return v;
}
#endif

}  // namespace rplu
