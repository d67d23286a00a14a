// FP32 operator kernels: the Jacobian apply used on the levels of the multigrid preconditioner.
#include <type_traits>
#include "op_launch.cuh"

namespace stmg {

template <>
cudaError_t launch_operator<float>(const Level& lv, const Problem& pb, int mode, double t0,
                                   const float* x, const float* state, const float* vprev,
                                   float* y, cudaStream_t s, int batch, int64_t xs, int64_t ys) {
  if (mode != OP_JAC) return cudaErrorNotSupported;   // residual and norms are FP64 only
  return launch_any<float, MJ>(lv, pb, t0, x, state, vprev, y, s, batch, xs, ys);
}

}  // namespace stmg
