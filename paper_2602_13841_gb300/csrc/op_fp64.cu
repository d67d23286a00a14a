// FP64 operator kernels: Jacobian apply and residual (outer Newton-Krylov level), and the
// nodal interpolation of the initial velocity.
#include <type_traits>
#include "op_launch.cuh"
#include "vec.cuh"

namespace stmg {

template <>
cudaError_t launch_operator<double>(const Level& lv, const Problem& pb, int mode, double t0,
                                    const double* x, const double* state, const double* vprev,
                                    double* y, cudaStream_t s, int batch, int64_t xs, int64_t ys) {
  if (mode == OP_RES) return launch_any<double, MR>(lv, pb, t0, x, state, vprev, y, s, batch, xs, ys);
  if (mode == OP_MASS) return launch_any<double, MM>(lv, pb, t0, x, state, vprev, y, s, batch, xs, ys);
  return launch_any<double, MJ>(lv, pb, t0, x, state, vprev, y, s, batch, xs, ys);
}

template <>
cudaError_t launch_level_residual<double>(const Level& lv, const Problem& pb, const double* rhs, const double* x,
                                       const double* state, double* y, cudaStream_t s, int columns, const double* nub) {
  cudaError_t e = launch_jac_tiled<double>(lv, pb, x, state, rhs, y, s, columns, nub);
  if (e != cudaErrorNotSupported) return e;
  e = launch_any<double, MJ>(lv, pb, 0.0, x, state, nullptr, y, s, columns, lv.Nst, lv.Nst, lv.Nst, nub);
  if (e == cudaSuccess && rhs) e = vaxpby<double>(columns * lv.Nst, 1.0, rhs, -1.0, y, s);
  return e;
}

// v_{0,h}: v0 evaluated at the mapped Gauss-Lobatto nodes (one thread per global node).
template <int D>
__global__ void k_initial(LevelArgs<double> L, Tab<double> tb, int r1, double* V0) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi >= L.nnodes) return;
  int gm[3] = {0, 0, 0};
  int64_t rem = gi;
  for (int l = 0; l < D; ++l) { gm[l] = (int)(rem % L.N1); rem /= L.N1; }
  int cc[3] = {0, 0, 0};
  double xh[3];
  for (int l = 0; l < D; ++l) {
    cc[l] = gm[l] / r1; if (cc[l] >= L.n) cc[l] = L.n - 1;
    xh[l] = tb.gll[gm[l] - cc[l] * r1];
  }
  double corner[8][3];
  for (int c = 0; c < (1 << D); ++c) {
    int64_t v = 0, s = 1;
    for (int l = 0; l < D; ++l) { v += (int64_t)(cc[l] + ((c >> l) & 1)) * s; s *= (L.n + 1); }
    for (int i = 0; i < D; ++i) corner[c][i] = L.verts[v * D + i];
  }
  double J[3][3], x[3], v0[3];
  map_jacobian<double, D>(corner, xh, J, x);
  problem_v0<D>(L.problem, x, L.nu, v0);
  for (int c = 0; c < D; ++c) V0[c * L.nnodes + gi] = v0[c];
}

cudaError_t launch_initial_condition(const Level& lv, const Problem& pb, double* V0, cudaStream_t s) {
  LevelArgs<double> L = level_args<double>(lv, pb, 0.0);
  Tab<double> tb = make_tab<double>(lv.tabs, pb.tau);
  int64_t blocks = (lv.nnodes + 255) / 256;
  if (lv.d == 2) k_initial<2><<<(unsigned)blocks, 256, 0, s>>>(L, tb, lv.r + 1, V0);
  else k_initial<3><<<(unsigned)blocks, 256, 0, s>>>(L, tb, lv.r + 1, V0);
  note_launch();
  return cudaGetLastError();
}

template <typename T, int N>
static void geo_launch(const Level& lv, const Problem& pb, T* geo, cudaStream_t s) {
  const int64_t ncells = (int64_t)lv.n * lv.n;
  int64_t blocks = (ncells * N * N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_geo2d<T, N><<<(unsigned)blocks, 256, 0, s>>>(level_args<T>(lv, pb, 0.0), make_tab<T>(lv.tabs, pb.tau), geo,
                                                 ncells);
  note_launch();
}

cudaError_t build_geometry(const Level& lv, const Problem& pb, cudaStream_t s) {
  if (lv.d != 2 || !lv.geo64 || !lv.geo32) return cudaErrorInvalidValue;
  const int N = lv.r + 2;
#define STMG_G(NN) { geo_launch<double, NN>(lv, pb, lv.geo64, s); geo_launch<float, NN>(lv, pb, lv.geo32, s); }
  if (N == 3) STMG_G(3) else if (N == 4) STMG_G(4) else if (N == 5) STMG_G(5) else return cudaErrorInvalidValue;
#undef STMG_G
  return cudaGetLastError();
}

}  // namespace stmg
