// Grid transfers between consecutive levels of the hp space-time hierarchy (Sec. 4.2).
//
// Prolongation P = E_time (x) P_space is the canonical embedding: a coarse function evaluated at
// the fine degrees of freedom.  Velocity: the global 1D operator P1 (coarse 1D Gauss-Lobatto
// Lagrange basis at the fine 1D node positions, reference-cell embedding of children) applied
// along each axis; pressure: coarse Legendre modes re-expanded exactly in the fine modes of
// each fine cell (per child type); time: E[i][j] = coarse Lagrange polynomial j at fine Radau
// point i.  Restriction is the exact transpose.  The level state is the fine velocity evaluated
// at the coarse nodes (I1 along each axis) and at the coarse Radau points (Et).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "level.hpp"

namespace stmg {

struct Csr1D {
  int rows = 0, cols = 0;
  int* rowptr = nullptr;   // device
  int* col = nullptr;
  double* val64 = nullptr;
  float* val32 = nullptr;
};

struct Transfer {
  const Level* fine = nullptr;
  const Level* coarse = nullptr;
  Csr1D P1, P1T, I1;
  double E[MAXKP1][MAXKP1]{};   // [kf+1][kc+1]
  double Et[MAXKP1][MAXKP1]{};  // [kc+1][kf+1]
  int ntypes = 1, ratio = 1;    // pressure child types (2^d for h-transfers)
  double* PT64 = nullptr;       // [ntypes][npf][npc]
  float* PT32 = nullptr;
  // scratch (element type of the preconditioner), `nb` slots of `scr` entries each
  void* tmpA = nullptr;
  void* tmpB = nullptr;
  void* tmpC = nullptr;
  int nb = 1;                   // slots: independent vectors transferred by one launch each
  int64_t scr = 0;

  // Each call transfers `slots` independent vectors (slot j at offset j * n_st of its level;
  // slots <= nb), in the same launches.
  template <typename T>
  cudaError_t prolong(const T* xc, T* xf, cudaStream_t s, int slots = 1) const;     // xf = P xc
  template <typename T>
  cudaError_t restrict_(const T* xf, T* xc, cudaStream_t s, int slots = 1) const;   // xc = P^T xf
  template <typename T>
  cudaError_t interp_state(const T* Vf, T* Vc, cudaStream_t s) const; // velocity part only, one slot
};

struct Handle;
// Build the transfer between levels[l] and levels[l+1]; scratch for element size `esize` and nb slots.
void build_transfer(Handle* h, Transfer& tr, const Level& fine, const Level& coarse, size_t esize, int nb = 1);

}  // namespace stmg
