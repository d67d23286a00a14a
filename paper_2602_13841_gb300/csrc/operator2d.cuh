// Warp-synchronous 2D volume kernel of the slab operator (Jacobian apply, residual, mass).
//
// Same arithmetic as k_volume (operator.cuh): per cell and time node, values at the Gauss points
// by two 1D passes with B, reference gradients by the collocation derivative Dc, quadrature
// point physics, integration by the transposed passes, temporal mixing with K^tau at the
// quadrature points.  Layout: Q = N^2 lanes per cell, floor(32 / Q) cells per warp; every 1D
// contraction is a set of register shuffles along the cell's lane rows / columns, so the
// kernel needs no shared memory and no block barrier.  Cells of one launch share no velocity
// node (colouring), so the scatter is race free and deterministic.
#pragma once
#include "operator.cuh"

namespace stmg {

template <typename T, int N>
__device__ __forceinline__ T shfl_x(T v, const T (*M)[MAXN], int row, int base, bool transpose) {
  // sum_j M[row][j] v(lane base + j)   (or M[j][row] when transposed); base = cell row start
  T acc = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T o = __shfl_sync(0xffffffffu, v, base + j);
    acc += (transpose ? M[j][row] : M[row][j]) * o;
  }
  return acc;
}

template <typename T, int N>
__device__ __forceinline__ T shfl_y(T v, const T (*M)[MAXN], int row, int base, bool transpose) {
  // sum_j M[row][j] v(lane base + j*N); base = cell start + column
  T acc = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T o = __shfl_sync(0xffffffffu, v, base + j * N);
    acc += (transpose ? M[j][row] : M[row][j]) * o;
  }
  return acc;
}

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(256) k_volume2d(OpArgs<T> A, Tab<T> tb, ColorInfo ci) {
  constexpr int Q = N * N;
  constexpr int CPW = 32 / Q;                       // cells per warp
  constexpr bool RES = (MODE == MR);
  constexpr bool MASS = (MODE == MM);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / Q;                        // cell slot inside the warp
  const int t = lane - slot * Q;                    // quadrature point / local node
  const int tx = t % N, ty = t / N;
  const int cb = slot * Q;                          // first lane of this cell
  const int cidx = (blockIdx.x * (blockDim.x >> 5) + warp) * CPW + slot;
  const bool on = (slot < CPW) && (cidx < ci.count);
  A.x += blockIdx.y * A.xs;
  A.y += blockIdx.y * A.ys;
  const LevelArgs<T>& L = A.L;
  const int kp1 = tb.k + 1, npc = tb.npc;
  int cc[3] = {0, 0, 0};
  if (on) decode_color_cell<2>(ci, cidx, cc);
  const int64_t gnode = on ? (int64_t)(cc[0] * (N - 1) + tx) + (int64_t)L.N1 * (cc[1] * (N - 1) + ty) : 0;
  const int64_t cell = (int64_t)cc[0] + (int64_t)L.n * cc[1];
  const int64_t poff = (int64_t)kp1 * L.Nv;

  // ---- loads (node values; lane t holds local node t)
  T dv[MAXKP1][2], st[MAXKP1][2], pm[MAXKP1], vp[2] = {0, 0};
#pragma unroll
  for (int b = 0; b < MAXKP1; ++b) {
    pm[b] = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      dv[b][c] = 0; st[b][c] = 0;
      if (on && b < kp1) {
        const int64_t gi = (int64_t)b * L.Nv + c * L.nnodes + gnode;
        dv[b][c] = A.x[gi];
        if (MODE == MJ) st[b][c] = A.state[gi];
      }
    }
    if (on && b < kp1 && t < npc) pm[b] = A.x[poff + (int64_t)b * L.Np + cell * npc + t];
  }
  if (RES && on)
    for (int c = 0; c < 2; ++c) vp[c] = A.vprev[c * L.nnodes + gnode];
  // corners and geometry at quadrature point t
  T corner[4][3];
  {
    const int64_t v0 = (int64_t)cc[0] + (int64_t)(L.n + 1) * cc[1];
    const int64_t vv[4] = {v0, v0 + 1, v0 + L.n + 1, v0 + L.n + 2};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int i = 0; i < 2; ++i) corner[q][i] = on ? L.verts[vv[q] * 2 + i] : (T)(((q >> i) & 1));
  }
  T G[3][3], xq[3], JxW;
  {
    T xh[3] = {tb.qx[tx], tb.qx[ty], 0}, J[3][3];
    map_jacobian<T, 2>(corner, xh, J, xq);
    JxW = invert<T, 2>(J, G) * tb.qw[tx] * tb.qw[ty];
  }
  // ---- node values -> quadrature values (two shuffle passes per array)
#pragma unroll
  for (int b = 0; b < MAXKP1; ++b)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (b < kp1) {
        T v = shfl_x<T, N>(dv[b][c], tb.B, tx, cb + ty * N, false);
        dv[b][c] = shfl_y<T, N>(v, tb.B, ty, cb + tx, false);
        if (MODE == MJ) {
          v = shfl_x<T, N>(st[b][c], tb.B, tx, cb + ty * N, false);
          st[b][c] = shfl_y<T, N>(v, tb.B, ty, cb + tx, false);
        }
      }
    }
  if (RES)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      T v = shfl_x<T, N>(vp[c], tb.B, tx, cb + ty * N, false);
      vp[c] = shfl_y<T, N>(v, tb.B, ty, cb + tx, false);
    }
  // pressure basis at this quadrature point
  T psi[MAXNP];
#pragma unroll
  for (int m = 0; m < MAXNP; ++m) psi[m] = (m < npc) ? tb.P1[tx][tb.modes[m][0]] * tb.P1[ty][tb.modes[m][1]] : (T)0;

  for (int a = 0; a < kp1; ++a) {
    // select time node a (registers are indexed statically)
    T dva[2], va[2], pma = 0;
#pragma unroll
    for (int b = 0; b < MAXKP1; ++b)
      if (b == a) {
        dva[0] = dv[b][0]; dva[1] = dv[b][1]; va[0] = st[b][0]; va[1] = st[b][1]; pma = pm[b];
      }
    if (MODE != MJ) { va[0] = dva[0]; va[1] = dva[1]; }
    // reference gradients by the collocation derivative
    T gref[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      gref[c][0] = shfl_x<T, N>(dva[c], tb.Dc, tx, cb + ty * N, false);
      gref[c][1] = shfl_y<T, N>(dva[c], tb.Dc, ty, cb + tx, false);
    }
    T pq = 0;
#pragma unroll
    for (int m = 0; m < MAXNP; ++m) {
      if (m < npc) pq += psi[m] * __shfl_sync(0xffffffffu, pma, cb + m);
    }
    T gp[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int l = 0; l < 2; ++l) gp[c][l] = G[0][l] * gref[c][0] + G[1][l] * gref[c][1];
    const T wa = tb.w[a];
    T Fh[2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      T F[2];
#pragma unroll
      for (int l = 0; l < 2; ++l) {
        T conv = RES ? va[c] * va[l] : dva[c] * va[l] + va[c] * dva[l];
        F[l] = MASS ? (T)0 : L.nu * gp[c][l] - conv - ((c == l) ? pq : (T)0);
      }
#pragma unroll
      for (int m = 0; m < 2; ++m) Fh[c][m] = wa * JxW * (G[m][0] * F[0] + G[m][1] * F[1]);
    }
    T fq[2] = {0, 0};
    if (RES && on) {
      double xd[3] = {(double)xq[0], (double)xq[1], 0.0}, fd[3];
      const double ta = (double)L.t0 + 0.5 * (double)L.tau * ((double)tb.that[a] + 1.0);
      problem_f<2>(L.problem, xd, ta, (double)L.nu, fd);
      fq[0] = (T)fd[0]; fq[1] = (T)fd[1];
    }
    T z[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      T acc = 0;
      if (MASS) {
        acc = wa * dva[c];
      } else {
#pragma unroll
        for (int b = 0; b < MAXKP1; ++b)
          if (b < kp1) acc += tb.K[a][b] * dv[b][c];
      }
      if (RES) acc -= tb.C[a] * vp[c] + wa * fq[c];
      z[c] = JxW * acc;
    }
    const T sp = MASS ? wa * JxW * pq : -wa * JxW * (gp[0][0] + gp[1][1]);
    // gradient test functions at the Gauss points (transposed collocation derivative)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      z[c] += shfl_x<T, N>(Fh[c][0], tb.Dc, tx, cb + ty * N, true);
      z[c] += shfl_y<T, N>(Fh[c][1], tb.Dc, ty, cb + tx, true);
    }
    // quadrature -> nodes (transposed B passes) and scatter
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      T v = shfl_x<T, N>(z[c], tb.B, tx, cb + ty * N, true);
      v = shfl_y<T, N>(v, tb.B, ty, cb + tx, true);
      if (on) A.y[(int64_t)a * L.Nv + c * L.nnodes + gnode] += v;
    }
    // pressure test functions: lane cb + m accumulates sum_t psi_m(t) sp(t)
    T pacc = 0;
    const int mo = t < npc ? t : 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      T s = __shfl_sync(0xffffffffu, sp, cb + q);
      pacc += tb.P1[q % N][tb.modes[mo][0]] * tb.P1[q / N][tb.modes[mo][1]] * s;
    }
    if (on && t < npc) A.y[poff + (int64_t)a * L.Np + cell * npc + t] += pacc;
  }
}

}  // namespace stmg
