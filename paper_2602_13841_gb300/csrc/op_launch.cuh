// Launch helpers for the operator kernels (included by the per-precision translation units).
#pragma once
#include <type_traits>
#include "level.hpp"
#include "operator.cuh"
#include "operator2d.cuh"
#include "operator2d_tile.cuh"
#include "counters.hpp"
#include <cstdlib>
#include <cstring>

namespace stmg {

template <typename T>
LevelArgs<T> level_args(const Level& lv, const Problem& pb, double t0) {
  LevelArgs<T> a{};
  a.verts = std::is_same<T, double>::value ? (const T*)lv.verts64 : (const T*)lv.verts32;
  a.n = lv.n; a.N1 = lv.N1;
  a.nnodes = lv.nnodes; a.Nv = lv.Nv; a.Np = lv.Np;
  a.nu = (T)pb.nu; a.gamma1 = (T)pb.gamma1; a.gamma2 = (T)pb.gamma2;
  a.hscale = (T)lv.hscale;
  a.bconv = pb.bconv; a.problem = pb.problem;
  a.t0 = (T)t0; a.tau = (T)pb.tau;
  a.ftab = pb.ftab; a.gtab = pb.gtab;
  return a;
}

template <typename T, int D, int N, int MODE>
static int vol_smem_per_cell(int kp1) {
  constexpr int Q = Shape<D, N>::Q;
  return ((MODE == MJ ? 3 : 2) * kp1 * D * Q + D * D * Q + 2 * D * Q + Q + kp1 * MAXNP + 8 * 3) * (int)sizeof(T);
}

template <typename T, int D, int N>
static int face_smem_per_cell(int kp1) {
  constexpr int Q = Shape<D, N>::Q;
  constexpr int NF = Shape<D, N>::NF;
  return (2 * kp1 * D * Q + kp1 * MAXNP + D * NF + D * D * NF + NF + Q + 4 + 8 * 3) * (int)sizeof(T);
}

template <typename T, int D, int N, int MODE>
static cudaError_t launch_dn(const Level& lv, const Problem& pb, double t0, const T* x,
                             const T* state, const T* vprev, T* y, cudaStream_t stream,
                             int batch, int64_t xs, int64_t ys, int64_t ss = 0, const T* nub = nullptr) {
  constexpr int Q = Shape<D, N>::Q;
  const int kp1 = lv.k + 1;
  Tab<T> tb = make_tab<T>(lv.tabs, pb.tau);
  const T* geo = nullptr;
  if constexpr (D == 2) {
    if constexpr (std::is_same<T, double>::value) geo = lv.geo64; else geo = lv.geo32;
  }
  OpArgs<T> A{level_args<T>(lv, pb, t0), x, state, vprev, y, xs, ys, geo, ss, nub};
  int cpb = 256 / Q; if (cpb < 1) cpb = 1;
  int smem = cpb * vol_smem_per_cell<T, D, N, MODE>(kp1);
  while (smem > 160 * 1024 && cpb > 1) { --cpb; smem = cpb * vol_smem_per_cell<T, D, N, MODE>(kp1); }
  cudaError_t e = allow_smem(k_volume<T, D, N, MODE>, (size_t)smem);
  if (e != cudaSuccess) return e;
  // faces: one boundary cell per block, so that the loop over the six faces skips the faces the
  // cell does not have (a block of several cells runs every face any of them has)
  int fcpb = 1;
  int fsmem = fcpb * face_smem_per_cell<T, D, N>(kp1);
  while (fsmem > 160 * 1024 && fcpb > 1) { --fcpb; fsmem = fcpb * face_smem_per_cell<T, D, N>(kp1); }
  if (MODE != MM) {
    e = allow_smem(k_faces<T, D, N, MODE>, (size_t)fsmem);
    if (e != cudaSuccess) return e;
  }
  for (int b = 0; b < batch; ++b) {
    e = cudaMemsetAsync(y + b * ys, 0, sizeof(T) * lv.Nst, stream);
    if (e != cudaSuccess) return e;
  }
  for (int c = 0; c < lv.ncolors; ++c) {
    const ColorInfo& ci = lv.colors[c];
    if (ci.count > 0) {
      if constexpr (D == 2) {
        // one group of Q lanes per (cell, time node)
        constexpr int cpw = 32 / Q, per_block = 8 * cpw;
        const int64_t groups = (int64_t)ci.count * kp1;
        dim3 grid((unsigned)((groups + per_block - 1) / per_block), batch);
        k_volume2d<T, N, MODE><<<grid, 256, 0, stream>>>(A, tb, ci);
      } else {
        dim3 grid((ci.count + cpb - 1) / cpb, batch);
        k_volume<T, D, N, MODE><<<grid, cpb * Q, smem, stream>>>(A, tb, ci, cpb);
      }
      note_launch();
    }
    if (D == 3 && MODE != MM && lv.nbcells[c] > 0) {       // 2D: faces fused into k_volume2d
      // one block per (boundary cell, time node) when fcpb == 1
      dim3 grid(fcpb == 1 ? lv.nbcells[c] * kp1 : (lv.nbcells[c] + fcpb - 1) / fcpb, batch);
      k_faces<T, D, N, MODE><<<grid, fcpb * Q, fsmem, stream>>>(A, tb, lv.bcells[c], lv.nbcells[c], fcpb);
      note_launch();
    }
  }
  return cudaGetLastError();
}

// Process-wide choice of the 2D Jacobian-apply kernel: the tiled single-launch kernel where it
// applies (default), or the colour-split warp kernel when the environment variable STMG_APPLY2D
// is "colour" (kept for comparisons; read once).
inline bool apply2d_tiled() {
  static const bool on = [] {
    const char* v = std::getenv("STMG_APPLY2D");
    return !(v && std::strcmp(v, "colour") == 0);
  }();
  return on;
}

template <typename T, int N>
static cudaError_t jac_tiled_n(const Level& lv, const Problem& pb, const T* x, const T* state, const T* rhs, T* y,
                               cudaStream_t s, int columns, const T* nub) {
  OpArgs<T> A{level_args<T>(lv, pb, 0.0), x, state, nullptr, y, lv.Nst, lv.Nst, nullptr, lv.Nst, nub};
  const Tab<T> tb = make_tab<T>(lv.tabs, pb.tau);
  cudaError_t e = cudaErrorNotSupported;
  if (lv.k == 0) e = launch_apply2d_tile<T, N, 1>(A, tb, rhs, lv.n, s, columns);
  else if (lv.k == 1) e = launch_apply2d_tile<T, N, 2>(A, tb, rhs, lv.n, s, columns);
  else if (lv.k == 2) e = launch_apply2d_tile<T, N, 3>(A, tb, rhs, lv.n, s, columns);
  if (e == cudaSuccess) note_launch();
  return e;
}

// y = J(state) x, or y = rhs - J(state) x when rhs is not null, by the tiled 2D kernel (one
// launch, y written without a zero fill).  `columns` independent applies at strides n_st (own
// increment, state, output and, with nub, viscosity).  cudaErrorNotSupported where it does not
// apply (3D, Q4/P3, FP64, or the colour kernels chosen).
template <typename T>
cudaError_t launch_jac_tiled(const Level& lv, const Problem& pb, const T* x, const T* state, const T* rhs, T* y,
                             cudaStream_t s, int columns = 1, const T* nub = nullptr) {
  if constexpr (!std::is_same<T, float>::value) {
    return cudaErrorNotSupported;
  } else {
    if (lv.d != 2 || !apply2d_tiled()) return cudaErrorNotSupported;
    if (lv.r == 1) return jac_tiled_n<T, 3>(lv, pb, x, state, rhs, y, s, columns, nub);
    if (lv.r == 2) return jac_tiled_n<T, 4>(lv, pb, x, state, rhs, y, s, columns, nub);
    return cudaErrorNotSupported;
  }
}

template <typename T, int MODE>
static cudaError_t launch_any(const Level& lv, const Problem& pb, double t0, const T* x,
                              const T* state, const T* vprev, T* y, cudaStream_t s,
                              int batch, int64_t xs, int64_t ys, int64_t ss = 0, const T* nub = nullptr) {
  const int N = lv.r + 2;
#define STMG_LAUNCH(DD, NN) return launch_dn<T, DD, NN, MODE>(lv, pb, t0, x, state, vprev, y, s, batch, xs, ys, ss, nub)
  if (lv.d == 2) {
    if (N == 3) STMG_LAUNCH(2, 3);
    if (N == 4) STMG_LAUNCH(2, 4);
    if (N == 5) STMG_LAUNCH(2, 5);
  } else {
    if (N == 3) STMG_LAUNCH(3, 3);
    if (N == 4) STMG_LAUNCH(3, 4);
    if (N == 5) STMG_LAUNCH(3, 5);
  }
#undef STMG_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace stmg
