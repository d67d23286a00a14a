// FP32 operator kernels: the Jacobian apply used on the levels of the multigrid preconditioner.
#include <type_traits>
#include "op_launch.cuh"

namespace stmg {

template <>
cudaError_t launch_operator<float>(const Level& lv, const Problem& pb, bool res, double t0,
                                   const float* x, const float* state, const float* vprev,
                                   float* y, cudaStream_t s) {
  if (res) return cudaErrorNotSupported;   // the residual is evaluated in FP64 only
  return launch_any<float, false>(lv, pb, t0, x, state, vprev, y, s);
}

}  // namespace stmg
