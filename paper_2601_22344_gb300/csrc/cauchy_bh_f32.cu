// Algorithm 3's kernels (cauchy_bh.cuh) instantiated for float data.
#include "cauchy_bh.cuh"

namespace rplu {

cudaError_t bh_run_f32(int32_t dtype, const CauchyLikeLaunch& a, const BhLaunch& b, cudaStream_t s, HotTimer* tm,
                       bool bounds_only) {
  return run_t<float>(dtype, a, b, s, tm, bounds_only);
}

}  // namespace rplu
