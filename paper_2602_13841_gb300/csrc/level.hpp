// Host-side description of one level of the hp space-time hierarchy and the operator launchers.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "refdata.hpp"

namespace stmg {

struct Level {
  int d = 2, n = 0, r = 1, k = 0;
  int N1 = 0, npc = 0;
  int64_t nnodes = 0, Nv = 0, Np = 0, Nst = 0;
  LevelTables tabs{};
  double* verts64 = nullptr;          // device, (n+1)^d * d
  float* verts32 = nullptr;
  ColorInfo colors[8]{};
  int* bcells[8]{};                   // device lists of boundary cells per colour
  int nbcells[8]{};
  int ncolors = 0;
  double hscale = 0;                  // Nitsche length factor (see LevelArgs)
  int64_t chunk_cells = 262144;       // cells per chunk of the smoother build's element scratch
  int smoother = 0;                   // 0: surrogate patches (Sec. 4.3); 1: diagonal space-time Vanka
  double* geo64 = nullptr;            // 2D: geometry table of the Jacobian apply (see OpArgs::geo)
  float* geo32 = nullptr;
};

struct Problem {
  double nu, tau, gamma1, gamma2;
  int bconv, problem;
  // STMG_USER: f at the volume Gauss points and g at the boundary-face Gauss points of the
  // finest level for the current slab (device tables filled from the host callbacks; see
  // LevelArgs::ftab / gtab for the layout)
  const double* ftab = nullptr;
  const double* gtab = nullptr;
};

template <typename T>
LevelArgs<T> level_args(const Level& lv, const Problem& pb, double t0);

enum OpMode { OP_JAC = 0, OP_RES = 1, OP_MASS = 2 };

// y = operator(x): J(state) x (OP_JAC), R(x; vprev) (OP_RES, FP64 only) or the slab mass
// diag(w_a M_h, w_a M_p) x (OP_MASS).  With batch > 1, column b reads x + b*xs and writes
// y + b*ys (the state is shared).  y is zeroed first.  Enqueued on `stream`.
template <typename T>
cudaError_t launch_operator(const Level& lv, const Problem& pb, int mode, double t0, const T* x,
                            const T* state, const T* vprev, T* y, cudaStream_t stream,
                            int batch = 1, int64_t xs = 0, int64_t ys = 0);

// y = rhs - J(state) x on a level (rhs null: y = J(state) x), the residual of a multigrid sweep;
// one launch where the tiled 2D kernel applies, else the operator followed by a vector update.
// `columns` independent residuals at strides n_st (own rhs, x, state, y; per-column viscosity
// nub[column] on the device, or null for pb.nu).
template <typename T>
cudaError_t launch_level_residual(const Level& lv, const Problem& pb, const T* rhs, const T* x, const T* state, T* y,
                                  cudaStream_t stream, int columns = 1, const T* nub = nullptr);

cudaError_t launch_initial_condition(const Level& lv, const Problem& pb, double* V0, cudaStream_t s);

// Fill lv.geo64 / lv.geo32 (allocated by the caller: cells x 5 x (r+2)^2 entries each) for a 2D
// level.
cudaError_t build_geometry(const Level& lv, const Problem& pb, cudaStream_t s);

}  // namespace stmg
