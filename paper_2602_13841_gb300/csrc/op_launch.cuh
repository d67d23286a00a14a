// Launch helpers for the operator kernels (included by the per-precision translation units).
#pragma once
#include "level.hpp"
#include "operator.cuh"

namespace stmg {

template <typename T>
LevelArgs<T> level_args(const Level& lv, const Problem& pb, double t0) {
  LevelArgs<T> a{};
  a.verts = std::is_same<T, double>::value ? (const T*)lv.verts64 : (const T*)lv.verts32;
  a.n = lv.n; a.N1 = lv.N1;
  a.nnodes = lv.nnodes; a.Nv = lv.Nv; a.Np = lv.Np;
  a.nu = (T)pb.nu; a.gamma1 = (T)pb.gamma1; a.gamma2 = (T)pb.gamma2;
  const int p = lv.r + 1;
  a.hfac = (T)(p * (p + 1));
  a.bconv = pb.bconv; a.problem = pb.problem;
  a.t0 = (T)t0; a.tau = (T)pb.tau;
  return a;
}

template <typename T, int D, int N, bool RES>
static int vol_smem_per_cell(int kp1) {
  constexpr int Q = Shape<D, N>::Q;
  return ((RES ? 2 : 3) * kp1 * D * Q + D * D * Q + 2 * D * Q + Q + kp1 * MAXNP + 8 * 3) * (int)sizeof(T);
}

template <typename T, int D, int N>
static int face_smem_per_cell(int kp1) {
  constexpr int Q = Shape<D, N>::Q;
  constexpr int NF = Shape<D, N>::NF;
  return (2 * kp1 * D * Q + kp1 * MAXNP + D * NF + D * D * NF + NF + Q + 4 + 8 * 3) * (int)sizeof(T);
}

template <typename T, int D, int N, bool RES>
static cudaError_t launch_dn(const Level& lv, const Problem& pb, double t0, const T* x,
                             const T* state, const T* vprev, T* y, cudaStream_t stream) {
  constexpr int Q = Shape<D, N>::Q;
  const int kp1 = lv.k + 1;
  Tab<T> tb = make_tab<T>(lv.tabs, pb.tau);
  OpArgs<T> A{level_args<T>(lv, pb, t0), x, state, vprev, y};
  int cpb = 256 / Q; if (cpb < 1) cpb = 1;
  int smem = cpb * vol_smem_per_cell<T, D, N, RES>(kp1);
  while (smem > 160 * 1024 && cpb > 1) { --cpb; smem = cpb * vol_smem_per_cell<T, D, N, RES>(kp1); }
  cudaError_t e = cudaFuncSetAttribute(k_volume<T, D, N, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int fcpb = 256 / Q; if (fcpb < 1) fcpb = 1;
  int fsmem = fcpb * face_smem_per_cell<T, D, N>(kp1);
  while (fsmem > 160 * 1024 && fcpb > 1) { --fcpb; fsmem = fcpb * face_smem_per_cell<T, D, N>(kp1); }
  e = cudaFuncSetAttribute(k_faces<T, D, N, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, fsmem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(y, 0, sizeof(T) * lv.Nst, stream);
  if (e != cudaSuccess) return e;
  for (int c = 0; c < lv.ncolors; ++c) {
    const ColorInfo& ci = lv.colors[c];
    if (ci.count > 0) {
      int blocks = (ci.count + cpb - 1) / cpb;
      k_volume<T, D, N, RES><<<blocks, cpb * Q, smem, stream>>>(A, tb, ci, cpb);
    }
    if (lv.nbcells[c] > 0) {
      int blocks = (lv.nbcells[c] + fcpb - 1) / fcpb;
      k_faces<T, D, N, RES><<<blocks, fcpb * Q, fsmem, stream>>>(A, tb, lv.bcells[c], lv.nbcells[c], fcpb);
    }
  }
  return cudaGetLastError();
}

template <typename T, bool RES>
static cudaError_t launch_any(const Level& lv, const Problem& pb, double t0, const T* x,
                              const T* state, const T* vprev, T* y, cudaStream_t s) {
  const int N = lv.r + 2;
  if (lv.d == 2) {
    if (N == 3) return launch_dn<T, 2, 3, RES>(lv, pb, t0, x, state, vprev, y, s);
    if (N == 4) return launch_dn<T, 2, 4, RES>(lv, pb, t0, x, state, vprev, y, s);
    if (N == 5) return launch_dn<T, 2, 5, RES>(lv, pb, t0, x, state, vprev, y, s);
  } else {
    if (N == 3) return launch_dn<T, 3, 3, RES>(lv, pb, t0, x, state, vprev, y, s);
    if (N == 4) return launch_dn<T, 3, 4, RES>(lv, pb, t0, x, state, vprev, y, s);
    if (N == 5) return launch_dn<T, 3, 5, RES>(lv, pb, t0, x, state, vprev, y, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace stmg
