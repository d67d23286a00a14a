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

constexpr int MAXNP2D = 10;   // C(r+2, 2) for r <= 3
// pressure modes of P_r on a level whose velocity has N = r + 2 nodes per direction: C(r+2, 2)
template <int N> __host__ __device__ constexpr int np2d() { return N * (N - 1) / 2; }

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

// Boundary-face terms of one face (axis, side) for time node a, added to the node outputs
// out[c] of lane (tx, ty) and to the pressure output pout of lane t = m (mode m).  Same
// integrand as k_faces (operator.cuh).  Face point p of face axis 0 is held by every lane of row
// ty = p (face axis 1: column tx = p); values at the face come from the GLL end-node row /
// column (L_j(side) = delta) followed by a 1D interpolation along the face; the normal reference
// derivative uses Dend.  All lanes of the warp execute this (shuffles), contributions of cells
// without this face are masked by `has`.
template <typename T, int N, int MODE>
__device__ __forceinline__ void face2d(const OpArgs<T>& A, const Tab<T>& tb, int a, int axis, int side, bool has,
                                       const T (*corner)[3], const int* cc, int64_t gnode, int64_t cell, int tx,
                                       int ty, int t, int cb, T vol, T* out, T& pout) {
  constexpr bool RES = (MODE == MR);
  const LevelArgs<T>& L = A.L;
  const T nu = column_nu(A);
  const int kp1 = tb.k + 1, npc = tb.npc;
  const int e = side * (N - 1);
  const int tn = axis == 0 ? tx : ty;           // lane index along the normal direction
  const int tt = axis == 0 ? ty : tx;           // lane index along the face (= face point p)
  // nodal values of the increment and of the state at this lane's node (time node a)
  T u[2] = {0, 0}, s[2] = {0, 0};
  if (has)
    for (int c = 0; c < 2; ++c) {
      const int64_t gi = (int64_t)a * L.Nv + c * L.nnodes + gnode;
      u[c] = A.x[gi];
      s[c] = (MODE == MJ) ? A.state[gi] : u[c];
    }
  const T pma = (has && t < npc) ? A.x[(int64_t)kp1 * L.Nv + (int64_t)a * L.Np + cell * npc + t] : (T)0;
  // end-node value and normal reference derivative on every lane of the face-parallel line
  T fv[2], fs[2], fdn[2], fdt[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T ve, vd, se;
    if (axis == 0) {
      ve = __shfl_sync(0xffffffffu, u[c], cb + ty * N + e);
      se = __shfl_sync(0xffffffffu, s[c], cb + ty * N + e);
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += tb.Dend[side][j] * __shfl_sync(0xffffffffu, u[c], cb + ty * N + j);
      vd = acc;
      // interpolate along y to face point p = ty
      fv[c] = shfl_y<T, N>(ve, tb.B, ty, cb + tx, false);
      fs[c] = shfl_y<T, N>(se, tb.B, ty, cb + tx, false);
      fdn[c] = shfl_y<T, N>(vd, tb.B, ty, cb + tx, false);
      fdt[c] = shfl_y<T, N>(ve, tb.D, ty, cb + tx, false);
    } else {
      ve = __shfl_sync(0xffffffffu, u[c], cb + e * N + tx);
      se = __shfl_sync(0xffffffffu, s[c], cb + e * N + tx);
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += tb.Dend[side][j] * __shfl_sync(0xffffffffu, u[c], cb + j * N + tx);
      vd = acc;
      fv[c] = shfl_x<T, N>(ve, tb.B, tx, cb + ty * N, false);
      fs[c] = shfl_x<T, N>(se, tb.B, tx, cb + ty * N, false);
      fdn[c] = shfl_x<T, N>(vd, tb.B, tx, cb + ty * N, false);
      fdt[c] = shfl_x<T, N>(ve, tb.D, tx, cb + ty * N, false);
    }
  }
  // pressure at face point tt: psi_m(face point) = Pend[side][m_axis] P1[tt][m_other]
  T fp = 0;
#pragma unroll
  for (int m = 0; m < np2d<N>(); ++m) {
    const T pm = __shfl_sync(0xffffffffu, pma, cb + m);
    const T psi = (axis == 0) ? tb.Pend[side][tb.modes[m][0]] * tb.P1[tt][tb.modes[m][1]]
                              : tb.P1[tt][tb.modes[m][0]] * tb.Pend[side][tb.modes[m][1]];
    fp += psi * pm;
  }
  // geometry at the face point
  T xh[3], J[3][3], G[3][3], xf[3];
  xh[axis] = (T)side;
  xh[1 - axis] = tb.qx[tt];
  xh[2] = 0;
  map_jacobian<T, 2>(corner, xh, J, xf);
  const T det = invert<T, 2>(J, G);
  const T nh = side ? (T)1 : (T)-1;
  T nrm[2], len2 = 0;
  for (int i = 0; i < 2; ++i) { nrm[i] = det * G[axis][i] * nh; len2 += nrm[i] * nrm[i]; }
  const T dS = sqrt(len2);
  nrm[0] /= dS; nrm[1] /= dS;
  const T JxWf = dS * tb.qw[tt];
  // face area (sum over the face points held by the lanes of one normal-direction column)
  T area = 0;
#pragma unroll
  for (int p = 0; p < N; ++p) area += __shfl_sync(0xffffffffu, JxWf, axis == 0 ? cb + p * N : cb + p);
  const T h = vol / area * L.hscale;
  // physical gradient of the increment and normal derivatives
  T dn[2];
  T ghat[2];
  for (int m = 0; m < 2; ++m) ghat[m] = G[m][0] * nrm[0] + G[m][1] * nrm[1];
  for (int c = 0; c < 2; ++c) {
    T gr[2];
    gr[axis] = fdn[c];
    gr[1 - axis] = fdt[c];
    T g0 = G[0][0] * gr[0] + G[1][0] * gr[1], g1 = G[0][1] * gr[0] + G[1][1] * gr[1];
    dn[c] = g0 * nrm[0] + g1 * nrm[1];
  }
  T y = fs[0] * nrm[0] + fs[1] * nrm[1];
  const T ypos = (T)0.5 * (fabs(y) + y), yneg = (T)0.5 * (fabs(y) - y);
  const T sgn = (y > 0) ? (T)1 : ((y < 0) ? (T)-1 : (T)0);
  T ev[2], gd[2] = {0, 0};
  if (RES) {
    double xd[3] = {(double)xf[0], (double)xf[1], 0.0}, gv[3];
    const double ta = (double)L.t0 + 0.5 * (double)L.tau * ((double)tb.that[a] + 1.0);
    if (L.problem == kProblemUser) {
      if (has) {
        const int64_t gb = ((((int64_t)a * 2 + axis) * 2 + side) * L.n + cc[1 - axis]) * 2 * N + tt;
        gv[0] = L.gtab[gb];
        gv[1] = L.gtab[gb + N];
      } else {
        gv[0] = gv[1] = 0.0;
      }
    } else {
      problem_g<2>(L.problem, xd, ta, (double)L.nu, gv);
    }
    gd[0] = (T)gv[0]; gd[1] = (T)gv[1];
    ev[0] = fs[0] - gd[0]; ev[1] = fs[1] - gd[1];
  } else {
    ev[0] = fv[0]; ev[1] = fv[1];
  }
  const T en = ev[0] * nrm[0] + ev[1] * nrm[1];
  const T gn = gd[0] * nrm[0] + gd[1] * nrm[1];
  const T wJ = has ? tb.w[a] * JxWf : (T)0;
  T ac[2], bg[2][2];
  for (int c = 0; c < 2; ++c) {
    T v = -nu * dn[c] + nu * L.gamma1 / h * ev[c] + L.gamma2 / h * en * nrm[c] + fp * nrm[c];
    if (L.bconv) {
      if (RES) v += (ypos - 2 * yneg) * fs[c] + (T)0.5 * (fabs(gn) - gn) * gd[c];
      else v += (ypos - 2 * yneg) * fv[c] + (T)0.5 * ((T)3 - sgn) * en * fs[c];
    }
    ac[c] = wJ * v;
    const T bc = -wJ * nu * ev[c];
    bg[c][0] = bc * ghat[0];
    bg[c][1] = bc * ghat[1];
  }
  const T sp = wJ * en;
  // test functions: node (tx, ty) gets
  //   [tn == e] (sum_p a(p) B[p][tt] + sum_p bg_t(p) D[p][tt]) + Dend[side][tn] sum_p bg_n(p) B[p][tt]
  for (int c = 0; c < 2; ++c) {
    T t1, t2, t3;
    if (axis == 0) {
      t1 = shfl_y<T, N>(ac[c], tb.B, ty, cb + tx, true);
      t2 = shfl_y<T, N>(bg[c][1], tb.D, ty, cb + tx, true);
      t3 = shfl_y<T, N>(bg[c][0], tb.B, ty, cb + tx, true);
    } else {
      t1 = shfl_x<T, N>(ac[c], tb.B, tx, cb + ty * N, true);
      t2 = shfl_x<T, N>(bg[c][0], tb.D, tx, cb + ty * N, true);
      t3 = shfl_x<T, N>(bg[c][1], tb.B, tx, cb + ty * N, true);
    }
    if (has) out[c] += (tn == e ? t1 + t2 : (T)0) + tb.Dend[side][tn] * t3;
  }
  // pressure test functions: lane m accumulates sum_p s(p) psi_m(p)
  const int mo = t < npc ? t : 0;
  T pa = 0;
#pragma unroll
  for (int p = 0; p < N; ++p) {
    const T sv = __shfl_sync(0xffffffffu, sp, axis == 0 ? cb + p * N : cb + p);
    const T psi = (axis == 0) ? tb.Pend[side][tb.modes[mo][0]] * tb.P1[p][tb.modes[mo][1]]
                              : tb.P1[p][tb.modes[mo][0]] * tb.Pend[side][tb.modes[mo][1]];
    pa += psi * sv;
  }
  if (has) pout += pa;
}

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_volume2d(OpArgs<T> A, Tab<T> tb, ColorInfo ci) {
  constexpr int Q = N * N;
  constexpr int CPW = 32 / Q;                       // (cell, time node) groups per warp
  constexpr bool RES = (MODE == MR);
  constexpr bool MASS = (MODE == MM);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / Q;                        // group slot inside the warp
  const int t = lane - slot * Q;                    // quadrature point / local node
  const int tx = t % N, ty = t / N;
  const int cb = slot * Q;                          // first lane of this group
  const int kp1 = tb.k + 1, npc = tb.npc;
  // 1D tables in shared memory: the passes index them by the lane's row (tx or ty), which
  // would serialise constant-bank reads of the kernel parameters
  __shared__ T sB[MAXN][MAXN], sDc[MAXN][MAXN], sP1[MAXN][4];
  for (int e = threadIdx.x; e < MAXN * MAXN; e += blockDim.x) {
    sB[e / MAXN][e % MAXN] = tb.B[e / MAXN][e % MAXN];
    sDc[e / MAXN][e % MAXN] = tb.Dc[e / MAXN][e % MAXN];
  }
  for (int e = threadIdx.x; e < MAXN * 4; e += blockDim.x) sP1[e / 4][e % 4] = tb.P1[e / 4][e % 4];
  __syncthreads();
  // one group of Q lanes per (cell, time node a): the time nodes of a cell couple only through
  // K^tau (and C^tau v_{n-1}), which is applied to the nodal values before the interpolation
  const int grp = (blockIdx.x * (blockDim.x >> 5) + warp) * CPW + slot;
  const int cidx = grp / kp1, a = grp - cidx * kp1;
  const bool on = (slot < CPW) && (cidx < ci.count);
  A.x += blockIdx.y * A.xs;
  A.y += blockIdx.y * A.ys;
  if (A.state) A.state += blockIdx.y * A.ss;
  const T nu = column_nu(A);
  const LevelArgs<T>& L = A.L;
  int cc[3] = {0, 0, 0};
  if (on) decode_color_cell<2>(ci, cidx, cc);
  const int64_t gnode = on ? (int64_t)(cc[0] * (N - 1) + tx) + (int64_t)L.N1 * (cc[1] * (N - 1) + ty) : 0;
  const int64_t cell = (int64_t)cc[0] + (int64_t)L.n * cc[1];
  const int64_t poff = (int64_t)kp1 * L.Nv;
  const T wa = tb.w[a];

  // ---- loads (node values; lane t holds local node t): the increment and the state at time
  // node a, and the time-mixed nodal vector u = sum_b K[a][b] x_b (- C[a] v_prev) or w_a x_a
  T dva[2] = {0, 0}, va[2] = {0, 0}, u[2] = {0, 0}, pma = 0;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    if (!on) continue;
    const int64_t gi = c * L.nnodes + gnode;
    dva[c] = A.x[(int64_t)a * L.Nv + gi];
    va[c] = (MODE == MJ) ? A.state[(int64_t)a * L.Nv + gi] : dva[c];
    T acc = 0;
    if (MASS) {
      acc = wa * dva[c];
    } else {
#pragma unroll
      for (int b = 0; b < MAXKP1; ++b)
        if (b < kp1) acc += tb.K[a][b] * (b == a ? dva[c] : A.x[(int64_t)b * L.Nv + gi]);
      if (RES) acc -= tb.C[a] * A.vprev[gi];
    }
    u[c] = acc;
  }
  if (on && t < npc) pma = A.x[poff + (int64_t)a * L.Np + cell * npc + t];
  // the output entries of this group (no other group of this colour writes them): read now, so
  // that the update at the end is a plain store
  T yold[2] = {0, 0}, pold = 0;
  if (on) {
#pragma unroll
    for (int c = 0; c < 2; ++c) yold[c] = A.y[(int64_t)a * L.Nv + c * L.nnodes + gnode];
    if (t < npc) pold = A.y[poff + (int64_t)a * L.Np + cell * npc + t];
  }
  // corners and geometry at quadrature point t: read from the precomputed table for the Jacobian
  // apply (the corners then only serve the boundary faces), else computed from the vertices
  const bool bcell = on && (cc[0] == 0 || cc[1] == 0 || cc[0] == L.n - 1 || cc[1] == L.n - 1);
  const bool use_geo = (MODE == MJ) && (A.geo != nullptr);
  T corner[4][3];
  {
    const bool need = use_geo ? bcell : on;
    const int64_t v0 = (int64_t)cc[0] + (int64_t)(L.n + 1) * cc[1];
    const int64_t vv[4] = {v0, v0 + 1, v0 + L.n + 1, v0 + L.n + 2};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int i = 0; i < 2; ++i) corner[q][i] = need ? L.verts[vv[q] * 2 + i] : (T)(((q >> i) & 1));
  }
  T G[3][3], xq[3] = {0, 0, 0}, JxW;
  if (use_geo) {
    const T* gg = A.geo + cell * 5 * Q + t;
    G[0][0] = on ? gg[0] : (T)1; G[0][1] = on ? gg[Q] : (T)0;
    G[1][0] = on ? gg[2 * Q] : (T)0; G[1][1] = on ? gg[3 * Q] : (T)1;
    JxW = on ? gg[4 * Q] : (T)0;
  } else {
    T xh[3] = {tb.qx[tx], tb.qx[ty], 0}, J[3][3];
    map_jacobian<T, 2>(corner, xh, J, xq);
    JxW = invert<T, 2>(J, G) * tb.qw[tx] * tb.qw[ty];
  }
  // ---- node values -> quadrature values (two shuffle passes per array)
  T dq[2], sq[2], uq[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T v = shfl_x<T, N>(dva[c], sB, tx, cb + ty * N, false);
    dq[c] = shfl_y<T, N>(v, sB, ty, cb + tx, false);
    if (MODE == MJ) {
      v = shfl_x<T, N>(va[c], sB, tx, cb + ty * N, false);
      sq[c] = shfl_y<T, N>(v, sB, ty, cb + tx, false);
    } else {
      sq[c] = dq[c];
    }
    v = shfl_x<T, N>(u[c], sB, tx, cb + ty * N, false);
    uq[c] = shfl_y<T, N>(v, sB, ty, cb + tx, false);
  }
  // cell volume |K| (for h_{Gamma_D} of boundary faces), needed only where a group has a face
  T vol = 0;
  if (MODE != MM && __any_sync(0xffffffffu, bcell)) {
#pragma unroll
    for (int q = 0; q < Q; ++q) vol += __shfl_sync(0xffffffffu, JxW, cb + q);
  }
  // pressure at this quadrature point
  T pq = 0;
#pragma unroll
  for (int m = 0; m < np2d<N>(); ++m) {
    const T pm = __shfl_sync(0xffffffffu, pma, cb + m);
    pq += sP1[tx][tb.modes[m][0]] * sP1[ty][tb.modes[m][1]] * pm;
  }
  // reference gradients by the collocation derivative of the Gauss-point values
  T gref[2][2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    gref[c][0] = shfl_x<T, N>(dq[c], sDc, tx, cb + ty * N, false);
    gref[c][1] = shfl_y<T, N>(dq[c], sDc, ty, cb + tx, false);
  }
  T gp[2][2];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int l = 0; l < 2; ++l) gp[c][l] = G[0][l] * gref[c][0] + G[1][l] * gref[c][1];
  T Fh[2][2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T F[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      T conv = RES ? sq[c] * sq[l] : dq[c] * sq[l] + sq[c] * dq[l];
      F[l] = MASS ? (T)0 : nu * gp[c][l] - conv - ((c == l) ? pq : (T)0);
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) Fh[c][m] = wa * JxW * (G[m][0] * F[0] + G[m][1] * F[1]);
  }
  T fq[2] = {0, 0};
  if (RES && on) {
    double xd[3] = {(double)xq[0], (double)xq[1], 0.0}, fd[3];
    const double ta = (double)L.t0 + 0.5 * (double)L.tau * ((double)tb.that[a] + 1.0);
    if (L.problem == kProblemUser) {
      const int64_t fb = (((int64_t)a * L.n * L.n + cell) * 2) * Q + t;
      fd[0] = L.ftab[fb];
      fd[1] = L.ftab[fb + Q];
    } else {
      problem_f<2>(L.problem, xd, ta, (double)L.nu, fd);
    }
    fq[0] = (T)fd[0]; fq[1] = (T)fd[1];
  }
  T z[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) z[c] = JxW * (uq[c] - (RES ? wa * fq[c] : (T)0));
  const T sp = MASS ? wa * JxW * pq : -wa * JxW * (gp[0][0] + gp[1][1]);
  // gradient test functions at the Gauss points (transposed collocation derivative)
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    z[c] += shfl_x<T, N>(Fh[c][0], sDc, tx, cb + ty * N, true);
    z[c] += shfl_y<T, N>(Fh[c][1], sDc, ty, cb + tx, true);
  }
  // quadrature -> nodes (transposed B passes)
  T vout[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T v = shfl_x<T, N>(z[c], sB, tx, cb + ty * N, true);
    vout[c] = shfl_y<T, N>(v, sB, ty, cb + tx, true);
  }
  // pressure test functions, sum_t psi_m(t) sp(t) with psi_m = P_mx(x) P_my(y), factorised:
  // lane (i, j) forms sum_qx P_i(qx) sp(qx, j), then sum_qy P_j(qy) of those along y; lane cb + m
  // takes the value of lane (mx, my).  Degrees run to r = N - 2; lanes i or j = N - 1 compute
  // an unused value (index clamped to a valid column of the table).
  const int dx = tx < N - 1 ? tx : 0, dy = ty < N - 1 ? ty : 0;
  T s1 = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) s1 += sP1[j][dx] * __shfl_sync(0xffffffffu, sp, cb + ty * N + j);
  T s2 = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) s2 += sP1[j][dy] * __shfl_sync(0xffffffffu, s1, cb + tx + j * N);
  const int mo = t < npc ? t : 0;
  T pacc = __shfl_sync(0xffffffffu, s2, cb + tb.modes[mo][0] + N * tb.modes[mo][1]);
  // boundary faces (Nitsche, boundary convection) of boundary cells
  if (MODE != MM) {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int axis = f >> 1, side = f & 1;
      const bool has = on && (side == 0 ? cc[axis] == 0 : cc[axis] == L.n - 1);
      if (__any_sync(0xffffffffu, has))
        face2d<T, N, MODE>(A, tb, a, axis, side, has, corner, cc, gnode, cell, tx, ty, t, cb, vol, vout, pacc);
    }
  }
  if (on) {
#pragma unroll
    for (int c = 0; c < 2; ++c) A.y[(int64_t)a * L.Nv + c * L.nnodes + gnode] = yold[c] + vout[c];
  }
  if (on && t < npc) A.y[poff + (int64_t)a * L.Np + cell * npc + t] = pold + pacc;
}

// Geometry table of a 2D level for k_volume2d: per cell and Gauss point t the inverse Jacobian
// G (dxhat_m/dx_l) and JxW of the multilinear map, computed exactly as in k_volume2d.
template <typename T, int N>
__global__ void k_geo2d(LevelArgs<T> L, Tab<T> tb, T* __restrict__ geo, int64_t ncells) {
  constexpr int Q = N * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ncells * Q;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = e / Q;
    const int t = (int)(e % Q), tx = t % N, ty = t / N;
    const int cx = (int)(cell % L.n), cy = (int)(cell / L.n);
    const int64_t v0 = (int64_t)cx + (int64_t)(L.n + 1) * cy;
    const int64_t vv[4] = {v0, v0 + 1, v0 + L.n + 1, v0 + L.n + 2};
    T corner[4][3];
    for (int q = 0; q < 4; ++q) {
      for (int i = 0; i < 2; ++i) corner[q][i] = L.verts[vv[q] * 2 + i];
      corner[q][2] = 0;
    }
    T xh[3] = {tb.qx[tx], tb.qx[ty], 0}, J[3][3], G[3][3], xq[3];
    map_jacobian<T, 2>(corner, xh, J, xq);
    const T JxW = invert<T, 2>(J, G) * tb.qw[tx] * tb.qw[ty];
    T* gg = geo + cell * 5 * Q + t;
    gg[0] = G[0][0]; gg[Q] = G[0][1]; gg[2 * Q] = G[1][0]; gg[3 * Q] = G[1][1]; gg[4 * Q] = JxW;
  }
}

}  // namespace stmg
