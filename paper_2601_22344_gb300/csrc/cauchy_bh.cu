// Algorithm 3 (Sec. 5.1) with the row draw by rejection sampling against the
// bounds of App. C: dispatch by data type to the translation units
// cauchy_bh_{f32,f64,c64,c128}.cu, which instantiate the kernels of
// cauchy_bh.cuh for one data type each.
#include "common.cuh"
#include "kernels.h"

namespace rplu {

cudaError_t bh_run_f32(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm,
                       bool bounds_only);
cudaError_t bh_run_f64(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm,
                       bool bounds_only);
cudaError_t bh_run_c64(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm,
                       bool bounds_only);
cudaError_t bh_run_c128(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm,
                        bool bounds_only);

namespace {

cudaError_t run_dt(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm,
                   bool bounds_only) {
  switch (dtype) {
    case RPLU_F32: return bh_run_f32(dtype, a, b, s, tm, bounds_only);
    case RPLU_F64: return bh_run_f64(dtype, a, b, s, tm, bounds_only);
    case RPLU_C64: return bh_run_c64(dtype, a, b, s, tm, bounds_only);
    case RPLU_C128: return bh_run_c128(dtype, a, b, s, tm, bounds_only);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t cauchy_like_bh_run(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s,
                               HotTimer* tm) {
  return run_dt(dtype, a, b, s, tm, false);
}

cudaError_t cauchy_like_bh_bounds(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s) {
  return run_dt(dtype, a, b, s, nullptr, true);
}

}  // namespace rplu
