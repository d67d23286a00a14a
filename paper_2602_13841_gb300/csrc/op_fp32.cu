// FP32 operator kernels: the Jacobian apply used on the levels of the multigrid preconditioner.
#include <type_traits>
#include "op_launch.cuh"
#include "vec.cuh"

namespace stmg {

template <>
cudaError_t launch_operator<float>(const Level& lv, const Problem& pb, int mode, double t0,
                                   const float* x, const float* state, const float* vprev,
                                   float* y, cudaStream_t s, int batch, int64_t xs, int64_t ys) {
  if (mode != OP_JAC) return cudaErrorNotSupported;   // residual and norms are FP64 only
  if (batch == 1) {
    cudaError_t e = launch_jac_tiled<float>(lv, pb, x, state, nullptr, y, s);
    if (e != cudaErrorNotSupported) return e;
  }
  return launch_any<float, MJ>(lv, pb, t0, x, state, vprev, y, s, batch, xs, ys);
}

template <>
cudaError_t launch_level_residual<float>(const Level& lv, const Problem& pb, const float* rhs, const float* x,
                                       const float* state, float* y, cudaStream_t s, int columns, const float* nub) {
  cudaError_t e = launch_jac_tiled<float>(lv, pb, x, state, rhs, y, s, columns, nub);
  if (e != cudaErrorNotSupported) return e;
  e = launch_any<float, MJ>(lv, pb, 0.0, x, state, nullptr, y, s, columns, lv.Nst, lv.Nst, lv.Nst, nub);
  if (e == cudaSuccess && rhs) e = vaxpby<float>(columns * lv.Nst, 1.0f, rhs, -1.0f, y, s);
  return e;
}

}  // namespace stmg
