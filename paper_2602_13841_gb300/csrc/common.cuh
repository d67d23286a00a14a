// Device-side common definitions: per-level tables, cell decoding, multilinear geometry and
// the analytic data of the bundled workloads.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "refdata.hpp"

namespace stmg {

// Per-level tables in the arithmetic type T (passed by value as a kernel parameter).
template <typename T>
struct Tab {
  T B[MAXN][MAXN];      // GLL Lagrange values at Gauss points  B[q][j]
  T D[MAXN][MAXN];      // GLL Lagrange derivatives at Gauss points
  T Dc[MAXN][MAXN];     // collocation derivative at Gauss points Dc[q][p]
  T Dend[2][MAXN];      // GLL Lagrange derivatives at x = 0, 1
  T P1[MAXN][4];        // Legendre P_i(2x-1) at Gauss points
  T Pend[2][4];         // Legendre at x = 0, 1
  T qx[MAXN], qw[MAXN], gll[MAXN];
  T K[MAXKP1][MAXKP1], w[MAXKP1], C[MAXKP1], phi_mid[MAXKP1], that[MAXKP1];
  signed char modes[MAXNP][3];
  int k, npc, r;
};

// Opt-in dynamic shared memory of a kernel.  The attribute belongs to the function and is shared
// by every handle in the process, so it is always set to the device maximum: a per-launch value
// would race between handles on different host threads (one thread lowering the cap between
// another thread's set and launch).  The cap is the opt-in maximum less the kernel's static
// shared memory; returns cudaErrorInvalidValue if `bytes` exceeds it.
template <typename F>
inline cudaError_t allow_smem(F* func, size_t bytes) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  const size_t cap = (size_t)optin - fa.sharedSizeBytes;     // static shared memory counts too
  if (bytes > cap) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
}

// Time diagonalisation of the Vanka patch for a slab of length tau (see LevelTables): block e
// has eigenvalue lam_e = (2/tau) mu_e of W^{-1} K, forward row F[e][a] = (2/tau) (Q^{-1}
// Omega^{-1})[e][a] and backward column G[a][e] (x2 for a complex block, whose conjugate
// partner is implied: y_a = sum_e Re(G[a][e] yhat_e)).
template <typename T>
struct TEig {
  int nblk;
  int cplx[MAXKP1], off[MAXKP1];
  T lre[MAXKP1], lim[MAXKP1];
  T Fre[MAXKP1][MAXKP1], Fim[MAXKP1][MAXKP1];
  T Gre[MAXKP1][MAXKP1], Gim[MAXKP1][MAXKP1];
};

template <typename T>
TEig<T> make_teig(const LevelTables& L, double tau) {
  TEig<T> t{};
  const double s = 2.0 / tau;
  t.nblk = L.tnblk;
  for (int b = 0; b < MAXKP1; ++b) {
    t.cplx[b] = L.tcplx[b]; t.off[b] = L.toff[b];
    t.lre[b] = (T)(s * L.tmu_re[b]); t.lim[b] = (T)(s * L.tmu_im[b]);
    for (int a = 0; a < MAXKP1; ++a) {
      t.Fre[b][a] = (T)(s * L.tF_re[b][a]); t.Fim[b][a] = (T)(s * L.tF_im[b][a]);
      t.Gre[a][b] = (T)L.tG_re[a][b]; t.Gim[a][b] = (T)L.tG_im[a][b];
    }
  }
  return t;
}

template <typename T>
Tab<T> make_tab(const LevelTables& L, double tau) {
  Tab<T> t{};
  for (int i = 0; i < MAXN; ++i)
    for (int j = 0; j < MAXN; ++j) {
      t.B[i][j] = (T)L.B[i][j]; t.D[i][j] = (T)L.D[i][j]; t.Dc[i][j] = (T)L.Dc[i][j];
    }
  for (int s = 0; s < 2; ++s) {
    for (int j = 0; j < MAXN; ++j) t.Dend[s][j] = (T)L.Dend[s][j];
    for (int i = 0; i < 4; ++i) t.Pend[s][i] = (T)L.Pend[s][i];
  }
  for (int q = 0; q < MAXN; ++q) {
    for (int i = 0; i < 4; ++i) t.P1[q][i] = (T)L.P1[q][i];
    t.qx[q] = (T)L.qx[q]; t.qw[q] = (T)L.qw[q]; t.gll[q] = (T)L.gll[q];
  }
  for (int a = 0; a < MAXKP1; ++a) {
    for (int b = 0; b < MAXKP1; ++b) t.K[a][b] = (T)L.K[a][b];
    t.w[a] = (T)(0.5 * tau * L.omega[a]);
    t.C[a] = (T)L.C[a];
    t.phi_mid[a] = (T)L.phi_mid[a];
    t.that[a] = (T)L.that[a];
  }
  for (int m = 0; m < MAXNP; ++m)
    for (int l = 0; l < 3; ++l) t.modes[m][l] = (signed char)L.modes[m][l];
  t.k = L.k; t.npc = L.npc; t.r = L.r;
  return t;
}

// Geometry / problem arguments shared by the operator kernels of one level.
template <typename T>
struct LevelArgs {
  const T* verts;      // (n+1)^d * d vertex coordinates, vertex-major
  int n, N1;
  int64_t nnodes, Nv, Np;
  T nu, gamma1, gamma2;
  // h_{Gamma_D} = |K| / |F| * hscale.  Finest level: hscale = 1 / (p (p+1)), p = r+1 (degree-scaled
  // interior-penalty length).  Coarser levels keep the finest level's penalty: hscale =
  // (n_level / n_finest) / (p0 (p0+1)), so the penalty term is the Galerkin product of the fine one.
  T hscale;
  int bconv, problem;
  T t0, tau;
  // STMG_USER data of the slab (finest level, residual only), time node a = 0..k:
  //   ftab[((a ncells + cell) D + c) Q + q]: f_c at Gauss point q (lexicographic, x fastest) of cell
  //   gtab[((((a D + axis) 2 + side) nf + f) D + c) NF + p]: g_c at face point p of the boundary
  //     face (axis, side) of the boundary cell whose other coordinates, lower axis fastest, give f
  //     (nf = n^(D-1)); face points lexicographic over the other axes, lower axis fastest
  const double* ftab;
  const double* gtab;
};

constexpr int kProblemUser = 5;   // STMG_USER

// Index of the boundary face (axis, side) of cell cc among the n^(D-1) faces of that side.
template <int D>
__device__ inline int64_t face_index(const int* cc, int axis, int n) {
  int64_t f = 0, s = 1;
  for (int l = 0; l < D; ++l)
    if (l != axis) { f += cc[l] * s; s *= n; }
  return f;
}

// Cells of one colour: coordinates of parity `color` (bit l = parity along axis l).
struct ColorInfo {
  int color;
  int cnt[3];   // number of cells of this colour along each axis
  int count;    // product
};

__host__ __device__ inline int ipow(int b, int e) { int r = 1; for (int i = 0; i < e; ++i) r *= b; return r; }

template <int D>
__device__ inline void decode_color_cell(const ColorInfo& ci, int idx, int* cc) {
  for (int l = 0; l < D; ++l) {
    int i = idx % ci.cnt[l];
    idx /= ci.cnt[l];
    cc[l] = 2 * i + ((ci.color >> l) & 1);
  }
}

// Multilinear map: Jacobian J[i][l] = dx_i / dxhat_l and the point x at reference point xh.
template <typename T, int D>
__device__ inline void map_jacobian(const T (*corner)[3], const T* xh, T (*J)[3], T* x) {
  for (int i = 0; i < D; ++i) { x[i] = 0; for (int l = 0; l < D; ++l) J[i][l] = 0; }
  for (int c = 0; c < (1 << D); ++c) {
    T N = 1, dN[3];
    for (int l = 0; l < D; ++l) dN[l] = 1;
    for (int l = 0; l < D; ++l) {
      int b = (c >> l) & 1;
      T val = b ? xh[l] : (T)1 - xh[l];
      T der = b ? (T)1 : (T)-1;
      N *= val;
      for (int g = 0; g < D; ++g) dN[g] *= (g == l) ? der : val;
    }
    for (int i = 0; i < D; ++i) {
      x[i] += corner[c][i] * N;
      for (int l = 0; l < D; ++l) J[i][l] += corner[c][i] * dN[l];
    }
  }
}

// G = J^{-1} (G[m][i] = dxhat_m/dx_i) and det J.
template <typename T, int D>
__device__ inline T invert(const T (*J)[3], T (*G)[3]) {
  if (D == 2) {
    T det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    T id = (T)1 / det;
    G[0][0] = J[1][1] * id; G[0][1] = -J[0][1] * id;
    G[1][0] = -J[1][0] * id; G[1][1] = J[0][0] * id;
    return det;
  } else {
    T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    T det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    T id = (T)1 / det;
    G[0][0] = c00 * id;
    G[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    G[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    G[1][0] = c01 * id;
    G[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    G[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    G[2][0] = c02 * id;
    G[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    G[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    return det;
  }
}

// ------------------------------------------------------------------ analytic data (double)
// TG2D: Taylor-Green vortex (exact solution, f = 0, g = v); MMS2D: manufactured solution of
// the convergence test (second component with a minus sign so that div v = 0), g = 0;
// TG3D: Taylor-Green initial field, g = v0, f = 0; MMS3D: sin t sin(pi z)(pi sin^2(pi x)
// sin(2 pi y), -pi sin(2 pi x) sin^2(pi y), 0) with p = sin t prod sin cos, g = 0; CAV3D: the
// lid-driven cavity of Sec. 5.2, g = (sin(pi t / 4), 0, 0) on the lid z = 1, zero on the other
// walls, f = 0, v0 = 0.  Face quadrature points are interior to their faces, so z = 1 (up to
// rounding of the multilinear map) holds exactly on the lid's points and nowhere else.
__device__ inline void problem_velocity_tg2d(const double* x, double t, double nu, double* v) {
  const double pi = 3.141592653589793238;
  double F = exp(-2.0 * pi * pi * nu * t);
  v[0] = F * sin(pi * x[0]) * cos(pi * x[1]);
  v[1] = -F * cos(pi * x[0]) * sin(pi * x[1]);
}

template <int D>
__device__ inline void problem_g(int problem, const double* x, double t, double nu, double* g) {
  const double pi = 3.141592653589793238;
  for (int i = 0; i < D; ++i) g[i] = 0.0;
  if (problem == 0 && D == 2) {
    problem_velocity_tg2d(x, t, nu, g);
  } else if (problem == 2 && D == 3) {
    g[0] = sin(pi * x[0]) * cos(pi * x[1]) * cos(pi * x[2]);
    g[1] = -cos(pi * x[0]) * sin(pi * x[1]) * cos(pi * x[2]);
  } else if (problem == 4 && D == 3) {
    if (x[2] > 1.0 - 1e-9) g[0] = sin(0.25 * pi * t);
  }
}

template <int D>
__device__ inline void problem_v0(int problem, const double* x, double nu, double* v) {
  problem_g<D>(problem, x, 0.0, nu, v);
}

template <int D>
__device__ inline void problem_f(int problem, const double* x, double t, double nu, double* f) {
  const double pi = 3.141592653589793238;
  for (int i = 0; i < D; ++i) f[i] = 0.0;
  double st = sin(t), ct = cos(t);
  if (problem == 1 && D == 2) {
    double sx = sin(pi * x[0]), cx = cos(pi * x[0]), sy = sin(pi * x[1]), cy = cos(pi * x[1]);
    double s2x = sin(2 * pi * x[0]), c2x = cos(2 * pi * x[0]);
    double s2y = sin(2 * pi * x[1]), c2y = cos(2 * pi * x[1]);
    double u = sx * sx * sy * cy, w = -sx * cx * sy * sy;          // spatial profile
    double ux = 2 * pi * sx * cx * sy * cy, uy = pi * sx * sx * c2y;
    double wx = -pi * c2x * sy * sy, wy = -2 * pi * sx * cx * sy * cy;
    double lu = 2 * pi * pi * c2x * sy * cy - 4 * pi * pi * sx * sx * sy * cy;
    double lw = 2 * pi * pi * s2x * sy * sy - 2 * pi * pi * sx * cx * c2y;
    double px = 0.5 * pi * c2x * s2y, py = 0.5 * pi * s2x * c2y;
    f[0] = ct * u + st * st * (u * ux + w * uy) - nu * st * lu + st * px;
    f[1] = ct * w + st * st * (u * wx + w * wy) - nu * st * lw + st * py;
  } else if (problem == 3 && D == 3) {
    double sx = sin(pi * x[0]), sy = sin(pi * x[1]);
    double s2x = sin(2 * pi * x[0]), c2x = cos(2 * pi * x[0]);
    double s2y = sin(2 * pi * x[1]), c2y = cos(2 * pi * x[1]);
    double s2z = sin(2 * pi * x[2]), c2z = cos(2 * pi * x[2]);
    double Z = sin(pi * x[2]);
    double a = pi * sx * sx * s2y, b = -pi * s2x * sy * sy;
    double ax = pi * pi * s2x * s2y, ay = 2 * pi * pi * sx * sx * c2y;
    double bx = -2 * pi * pi * c2x * sy * sy, by = -pi * pi * s2x * s2y;
    double la = 2 * pi * pi * pi * c2x * s2y - 4 * pi * pi * pi * sx * sx * s2y - pi * pi * a;
    double lb = 4 * pi * pi * pi * s2x * sy * sy - 2 * pi * pi * pi * s2x * c2y - pi * pi * b;
    double v1 = Z * a, v2 = Z * b;                                   // spatial profile
    double g1x = Z * ax, g1y = Z * ay;                               // d/dz terms meet v3 = 0
    double g2x = Z * bx, g2y = Z * by;
    double px = 0.25 * pi * c2x * s2y * s2z, py = 0.25 * pi * s2x * c2y * s2z, pz = 0.25 * pi * s2x * s2y * c2z;
    f[0] = ct * v1 + st * st * (v1 * g1x + v2 * g1y) - nu * st * Z * la + st * px;
    f[1] = ct * v2 + st * st * (v1 * g2x + v2 * g2y) - nu * st * Z * lb + st * py;
    f[2] = st * pz;
  }
}

}  // namespace stmg
