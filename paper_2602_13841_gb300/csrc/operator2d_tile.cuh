// Tiled 2D Jacobian apply: y = J_n(U) x, or y = rhs - J_n(U) x (the level residual of a
// multigrid sweep), in one launch per apply.
//
// Same discrete operator as k_volume2d / k_faces (Sec. 4.4, Eq. JacobianLocal0-1): per cell and
// time node a, the increment, the state and the time-mixed increment u_a = sum_b K_ab x_b are
// interpolated to the Gauss points by two 1D passes, reference gradients are taken by the
// collocation derivative, the flux of the linearised convection, viscosity and pressure is
// formed pointwise, and the transposed passes integrate against the test functions; boundary
// cells add the Nitsche / boundary-convection face terms.
//
// GB300 layout.  One thread owns one cell and loops over the time nodes; every 1D contraction
// runs on registers with the reference tables as compile-time-indexed kernel-parameter
// operands (no shuffles, no shared-memory traffic inside a pass).  A block computes a tile of
// CX x CY cells whose node values (increment and state at every time node) are staged in shared
// memory by coalesced asynchronous copies; u_a is formed from the staged increments while they
// are interpolated.  The tile reaches one cell beyond its owned
// cells on the low side in x and y; every node the tile owns then receives the contributions of
// all its cells inside the block, summed in shared memory in a fixed order (the four parity
// classes of the cells one after another), so y is written once, with plain coalesced stores,
// without atomics and without a zero fill: the result is deterministic.
#pragma once
#include "operator.cuh"

namespace stmg {

template <int N>
struct Tile2D {
  static constexpr int CX = 16, CY = 8;              // computed cells (incl. the low halo)
  static constexpr int THREADS = CX * CY;
  static constexpr int NX = CX * (N - 1) + 1, NY = CY * (N - 1) + 1, NXY = NX * NY;
};

// Pressure mode m of P_r in 2D (total degree, then ascending y degree): x and y degrees.
__host__ __device__ constexpr int mode2d_x(int m) {
  int s = 0;
  while (m > s) { m -= s + 1; ++s; }
  return s - m;
}
__host__ __device__ constexpr int mode2d_y(int m) {
  int s = 0;
  while (m > s) { m -= s + 1; ++s; }
  return m;
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gsrc, bool valid) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  const int n = valid ? (int)sizeof(T) : 0;          // src-size 0: the element is zero filled
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gsrc), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ T rcp_t(T v) { return (T)1 / v; }
template <>
__device__ __forceinline__ float rcp_t<float>(float v) { return __fdividef(1.0f, v); }

// Sum-factorised interpolation of the N x N nodal values of one component (node (i, j) at
// src[i + NX j]) to the Gauss points: out[qy * N + qx].
template <typename T, int N, int NX>
__device__ __forceinline__ void interp2(const T* __restrict__ src, const Tab<T>& tb, T* out) {
  T t[N][N];                                          // t[j][qx]: x pass of row j
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = src[i + NX * j];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T acc = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) acc += tb.B[q][i] * v[i];
      t[j][q] = acc;
    }
  }
#pragma unroll
  for (int qy = 0; qy < N; ++qy)
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += tb.B[qy][j] * t[j][qx];
      out[qy * N + qx] = acc;
    }
}

// The same for the time-mixed nodal values u_a = sum_b K_ab x_b (node (i, j) of time node b at
// src[b * bstride + i + NX j]).
template <typename T, int N, int NX, int KP1>
__device__ __forceinline__ void interp2_mixed(const T* __restrict__ src, int bstride, const T* Ka,
                                              const Tab<T>& tb, T* out) {
  T t[N][N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T acc = 0;
#pragma unroll
      for (int b = 0; b < KP1; ++b) acc += Ka[b] * src[b * bstride + i + NX * j];
      v[i] = acc;
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T acc = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) acc += tb.B[q][i] * v[i];
      t[j][q] = acc;
    }
  }
#pragma unroll
  for (int qy = 0; qy < N; ++qy)
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += tb.B[qy][j] * t[j][qx];
      out[qy * N + qx] = acc;
    }
}

// Boundary face (axis, side) of one cell at time node a, Jacobian form (Eq. def-b-gam, Defcp,
// bttp linearised): adds the test-function integrals to out (nodal, [c][j*N+i]) and pacc.
template <typename T, int N, int NX, int NPC>
__device__ __forceinline__ void face_jac_tile(const Tab<T>& tb, const LevelArgs<T>& L, int axis, int side,
                                              const T* __restrict__ xs0, const T* __restrict__ xs1,
                                              const T* __restrict__ ss0, const T* __restrict__ ss1,
                                              const T* pm, const T (&gc)[6], T vol, T wa, T nu,
                                              T (&out)[2][N * N], T (&pacc)[NPC]) {
  const int e = side * (N - 1);
  const T* xsc[2] = {xs0, xs1};
  const T* ssc[2] = {ss0, ss1};
  // nodal values on the face line (end node of every line normal to the face), the normal
  // reference derivative there, and the state on the face line
  T ve[2][N], vd[2][N], se[2][N];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int t = 0; t < N; ++t) {
      const int ie = axis == 0 ? e + NX * t : t + NX * e;
      ve[c][t] = xsc[c][ie];
      se[c][t] = ssc[c][ie];
      T acc = 0;
#pragma unroll
      for (int m = 0; m < N; ++m) acc += tb.Dend[side][m] * xsc[c][axis == 0 ? m + NX * t : t + NX * m];
      vd[c][t] = acc;
    }
  const T ax = gc[0], bx = gc[1], cx = gc[2], ay = gc[3], by = gc[4], cy = gc[5];
  const T nh = side ? (T)1 : (T)-1;
  // face points: geometry first (the face area enters h_{Gamma_D})
  T nrm[N][2], dS[N], G[N][2][2];
  T area = 0;
#pragma unroll
  for (int p = 0; p < N; ++p) {
    const T xi = axis == 0 ? (T)side : tb.qx[p];
    const T eta = axis == 0 ? tb.qx[p] : (T)side;
    const T J00 = ax + cx * eta, J01 = bx + cx * xi, J10 = ay + cy * eta, J11 = by + cy * xi;
    const T det = J00 * J11 - J01 * J10;
    const T id = rcp_t<T>(det);
    G[p][0][0] = J11 * id; G[p][0][1] = -J01 * id; G[p][1][0] = -J10 * id; G[p][1][1] = J00 * id;
    T n0 = axis == 0 ? J11 * nh : -J10 * nh;          // det G[axis][:] * nh
    T n1 = axis == 0 ? -J01 * nh : J00 * nh;
    const T s = sqrt(n0 * n0 + n1 * n1);
    const T is = rcp_t<T>(s);
    nrm[p][0] = n0 * is; nrm[p][1] = n1 * is;
    dS[p] = s;
    area += s * tb.qw[p];
  }
  const T h = vol / area * L.hscale;
  const T pen1 = nu * L.gamma1 / h, pen2 = L.gamma2 / h;
  T tA[2][N], tB[2][N];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int t = 0; t < N; ++t) { tA[c][t] = 0; tB[c][t] = 0; }
  T spp[N];
#pragma unroll
  for (int p = 0; p < N; ++p) {
    T fv[2], fs[2], fdn[2], fdt[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
      for (int t = 0; t < N; ++t) {
        a0 += tb.B[p][t] * ve[c][t];
        a1 += tb.B[p][t] * se[c][t];
        a2 += tb.B[p][t] * vd[c][t];
        a3 += tb.D[p][t] * ve[c][t];
      }
      fv[c] = a0; fs[c] = a1; fdn[c] = a2; fdt[c] = a3;
    }
    T fp = 0;
#pragma unroll
    for (int m = 0; m < NPC; ++m) {
      const T psi = axis == 0 ? tb.Pend[side][mode2d_x(m)] * tb.P1[p][mode2d_y(m)]
                              : tb.P1[p][mode2d_x(m)] * tb.Pend[side][mode2d_y(m)];
      fp += psi * pm[m];
    }
    const T n0 = nrm[p][0], n1 = nrm[p][1];
    T dn[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T gr0 = axis == 0 ? fdn[c] : fdt[c], gr1 = axis == 0 ? fdt[c] : fdn[c];
      const T g0 = G[p][0][0] * gr0 + G[p][1][0] * gr1, g1 = G[p][0][1] * gr0 + G[p][1][1] * gr1;
      dn[c] = g0 * n0 + g1 * n1;
    }
    const T gh0 = G[p][0][0] * n0 + G[p][0][1] * n1, gh1 = G[p][1][0] * n0 + G[p][1][1] * n1;
    const T y = fs[0] * n0 + fs[1] * n1;
    const T ypos = (T)0.5 * (fabs(y) + y), yneg = (T)0.5 * (fabs(y) - y);
    const T sgn = (y > 0) ? (T)1 : ((y < 0) ? (T)-1 : (T)0);
    const T en = fv[0] * n0 + fv[1] * n1;
    const T wJ = wa * dS[p] * tb.qw[p];
    T ac[2], bgn[2], bgt[2];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T nc = c == 0 ? n0 : n1;
      T v = -nu * dn[c] + pen1 * fv[c] + pen2 * en * nc + fp * nc;
      if (L.bconv) v += (ypos - 2 * yneg) * fv[c] + (T)0.5 * ((T)3 - sgn) * en * fs[c];
      ac[c] = wJ * v;
      const T bc = -wJ * nu * fv[c];
      bgn[c] = bc * (axis == 0 ? gh0 : gh1);            // normal reference direction
      bgt[c] = bc * (axis == 0 ? gh1 : gh0);            // along the face
    }
    spp[p] = wJ * en;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int t = 0; t < N; ++t) {
        tA[c][t] += ac[c] * tb.B[p][t] + bgt[c] * tb.D[p][t];
        tB[c][t] += bgn[c] * tb.B[p][t];
      }
  }
  // node (i, j): [normal index == e] tA(t) + Dend[side][normal index] tB(t), t = index along the face
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int tn = axis == 0 ? i : j, tt = axis == 0 ? j : i;
        T v = tb.Dend[side][tn] * tB[c][tt];
        if (tn == e) v += tA[c][tt];
        out[c][j * N + i] += v;
      }
#pragma unroll
  for (int m = 0; m < NPC; ++m) {
    T acc = 0;
#pragma unroll
    for (int p = 0; p < N; ++p) {
      const T psi = axis == 0 ? tb.Pend[side][mode2d_x(m)] * tb.P1[p][mode2d_y(m)]
                              : tb.P1[p][mode2d_x(m)] * tb.Pend[side][mode2d_y(m)];
      acc += psi * spp[p];
    }
    pacc[m] += acc;
  }
}

template <typename T, int N, int KP1>
__global__ void __launch_bounds__(Tile2D<N>::THREADS, 3)
k_apply2d_tile(OpArgs<T> A, Tab<T> tb, const T* __restrict__ rhs, int tiles_x) {
  using TL = Tile2D<N>;
  constexpr int CX = TL::CX, CY = TL::CY, NX = TL::NX, NY = TL::NY, NXY = TL::NXY;
  constexpr int Q = N * N;
  constexpr int R = N - 2;
  constexpr int NPC = (R + 1) * (R + 2) / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);               // [KP1][2][NXY] increment
  T* ss = xs + KP1 * 2 * NXY;                        // [KP1][2][NXY] state
  const LevelArgs<T>& L = A.L;
  // blockIdx.y: independent column of a batched apply (own increment, state, output, viscosity)
  A.x += blockIdx.y * A.xs;
  A.state += blockIdx.y * A.ss;
  A.y += blockIdx.y * A.ys;
  if (rhs) rhs += blockIdx.y * A.ys;
  const int n = L.n, N1 = L.N1;
  const int tix = blockIdx.x % tiles_x, tiy = blockIdx.x / tiles_x;
  const int cx0 = tix * (CX - 1) - 1, cy0 = tiy * (CY - 1) - 1;   // first computed cell
  const int X0 = cx0 * (N - 1), Y0 = cy0 * (N - 1);                // first tile node
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = TL::THREADS / 32;

  // ---- stage the node values of the tile (zero outside the mesh): one warp per tile row
  for (int row = warp; row < KP1 * 2 * NY; row += NW) {
    const int arr = row / NY, iy = row - arr * NY;
    const int gy = Y0 + iy;
    const bool vy = gy >= 0 && gy < N1;
    const int64_t gb = (int64_t)(arr >> 1) * L.Nv + (int64_t)(arr & 1) * L.nnodes + (int64_t)gy * N1 + X0;
    T* dx = xs + arr * NXY + iy * NX;
    T* ds = ss + arr * NXY + iy * NX;
    for (int ix = lane; ix < NX; ix += 32) {
      const int gx = X0 + ix;
      const bool valid = vy && gx >= 0 && gx < N1;
      cp_async_elem<T>(dx + ix, valid ? A.x + gb + ix : A.x, valid);
      cp_async_elem<T>(ds + ix, valid ? A.state + gb + ix : A.state, valid);
    }
  }
  // this thread's cell, its corners and the bilinear map coefficients
  const int lcx = tid % CX, lcy = tid / CX;
  const int cx = cx0 + lcx, cy = cy0 + lcy;
  const bool on = cx >= 0 && cx < n && cy >= 0 && cy < n;
  T gc[6] = {1, 0, 0, 0, 1, 0};                      // ax, bx, cx, ay, by, cy
  if (on) {
    const int64_t v0 = (int64_t)cx + (int64_t)(n + 1) * cy;
    const T x0 = L.verts[2 * v0], y0 = L.verts[2 * v0 + 1];
    const T x1 = L.verts[2 * (v0 + 1)], y1 = L.verts[2 * (v0 + 1) + 1];
    const T x2 = L.verts[2 * (v0 + n + 1)], y2 = L.verts[2 * (v0 + n + 1) + 1];
    const T x3 = L.verts[2 * (v0 + n + 2)], y3 = L.verts[2 * (v0 + n + 2) + 1];
    gc[0] = x1 - x0; gc[1] = x2 - x0; gc[2] = x3 - x2 - x1 + x0;
    gc[3] = y1 - y0; gc[4] = y2 - y0; gc[5] = y3 - y2 - y1 + y0;
  }
  // det J of a bilinear map is affine in the reference point: d0 + d1 xi + d2 eta
  const T d0 = gc[0] * gc[4] - gc[1] * gc[3];
  const T d1 = gc[0] * gc[5] - gc[2] * gc[3];
  const T d2 = gc[2] * gc[4] - gc[1] * gc[5];
  const T vol = d0 + (T)0.5 * (d1 + d2);
  const int64_t cell = (int64_t)cx + (int64_t)n * cy;
  const int64_t poff = (int64_t)KP1 * L.Nv;
  const bool bcell = on && (cx == 0 || cy == 0 || cx == n - 1 || cy == n - 1);
  cp_async_wait_all();
  __syncthreads();

  const int nb = lcx * (N - 1) + NX * (lcy * (N - 1));   // the cell's first node in the tile
  const T nu = column_nu(A);
#pragma unroll 1
  for (int a = 0; a < KP1; ++a) {
    const T wa = tb.w[a];
    T* xa0 = xs + (a * 2) * NXY + nb;
    T* xa1 = xa0 + NXY;
    const T* sa0 = ss + (a * 2) * NXY + nb;
    const T* sa1 = sa0 + NXY;
    T out[2][Q];
    T pacc[NPC];
#pragma unroll
    for (int m = 0; m < NPC; ++m) pacc[m] = 0;
    if (on) {
      // mass term sum_b K_ab M_K x_b at the Gauss points: z = JxW u_a (the staged increments of
      // every time node stay in place for the whole tile; outputs go to the state buffers)
      T z[2][Q];
      T Ka[KP1];
#pragma unroll
      for (int b = 0; b < KP1; ++b) Ka[b] = tb.K[a][b];
      interp2_mixed<T, N, NX, KP1>(xs + nb, 2 * NXY, Ka, tb, z[0]);
      interp2_mixed<T, N, NX, KP1>(xs + NXY + nb, 2 * NXY, Ka, tb, z[1]);
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          const T jw = (d0 + d1 * tb.qx[qx] + d2 * tb.qx[qy]) * (tb.qw[qx] * tb.qw[qy]);
          z[0][qy * N + qx] *= jw;
          z[1][qy * N + qx] *= jw;
        }
      T dq[2][Q], sq[2][Q];
      interp2<T, N, NX>(xa0, tb, dq[0]);
      interp2<T, N, NX>(xa1, tb, dq[1]);
      interp2<T, N, NX>(sa0, tb, sq[0]);
      interp2<T, N, NX>(sa1, tb, sq[1]);
      // pressure modes of this cell and time node; ry[my][qx] = sum_mx P_mx(qx) p_(mx,my)
      T pm[NPC];
#pragma unroll
      for (int m = 0; m < NPC; ++m) pm[m] = A.x[poff + (int64_t)a * L.Np + cell * NPC + m];
      T ry[R + 1][N];
#pragma unroll
      for (int my = 0; my <= R; ++my)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          T acc = 0;
#pragma unroll
          for (int m = 0; m < NPC; ++m)
            if (mode2d_y(m) == my) acc += tb.P1[qx][mode2d_x(m)] * pm[m];
          ry[my][qx] = acc;
        }
      // pointwise fluxes, row by row of Gauss points
#pragma unroll
      for (int qy = 0; qy < N; ++qy) {
        T sx[R + 1];
#pragma unroll
        for (int mx = 0; mx <= R; ++mx) sx[mx] = 0;
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          const int q = qy * N + qx;
          const T xi = tb.qx[qx], eta = tb.qx[qy];
          const T J00 = gc[0] + gc[2] * eta, J01 = gc[1] + gc[2] * xi;
          const T J10 = gc[3] + gc[5] * eta, J11 = gc[4] + gc[5] * xi;
          const T det = d0 + d1 * xi + d2 * eta;
          const T id = rcp_t<T>(det);
          const T G00 = J11 * id, G01 = -J01 * id, G10 = -J10 * id, G11 = J00 * id;
          const T wJ = wa * det * (tb.qw[qx] * tb.qw[qy]);
          T pq = 0;
#pragma unroll
          for (int my = 0; my <= R; ++my) pq += tb.P1[qy][my] * ry[my][qx];
          T gp[2][2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            T g0 = 0, g1 = 0;
#pragma unroll
            for (int j = 0; j < N; ++j) {
              g0 += tb.Dc[qx][j] * dq[c][qy * N + j];
              g1 += tb.Dc[qy][j] * dq[c][j * N + qx];
            }
            gp[c][0] = G00 * g0 + G10 * g1;
            gp[c][1] = G01 * g0 + G11 * g1;
          }
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            T F[2];
#pragma unroll
            for (int l = 0; l < 2; ++l)
              F[l] = nu * gp[c][l] - (dq[c][q] * sq[l][q] + sq[c][q] * dq[l][q]) - (c == l ? pq : (T)0);
            const T Fh0 = wJ * (G00 * F[0] + G01 * F[1]);
            const T Fh1 = wJ * (G10 * F[0] + G11 * F[1]);
            // gradient test functions: transposed collocation derivative along x and y
#pragma unroll
            for (int j = 0; j < N; ++j) {
              z[c][qy * N + j] += tb.Dc[qx][j] * Fh0;
              z[c][j * N + qx] += tb.Dc[qy][j] * Fh1;
            }
          }
          const T sp = -wJ * (gp[0][0] + gp[1][1]);
#pragma unroll
          for (int mx = 0; mx <= R; ++mx) sx[mx] += tb.P1[qx][mx] * sp;
        }
#pragma unroll
        for (int m = 0; m < NPC; ++m) pacc[m] += tb.P1[qy][mode2d_y(m)] * sx[mode2d_x(m)];
      }
      // quadrature -> nodes: transposed B passes
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        T t[N][N];                                     // t[qy][i]
#pragma unroll
        for (int qy = 0; qy < N; ++qy)
#pragma unroll
          for (int i = 0; i < N; ++i) {
            T acc = 0;
#pragma unroll
            for (int qx = 0; qx < N; ++qx) acc += tb.B[qx][i] * z[c][qy * N + qx];
            t[qy][i] = acc;
          }
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
          for (int i = 0; i < N; ++i) {
            T acc = 0;
#pragma unroll
            for (int qy = 0; qy < N; ++qy) acc += tb.B[qy][j] * t[qy][i];
            out[c][j * N + i] = acc;
          }
      }
      if (bcell) {
#pragma unroll 1
        for (int f = 0; f < 4; ++f) {
          const int axis = f >> 1, side = f & 1;
          const int cc = axis == 0 ? cx : cy;
          if (side == 0 ? cc == 0 : cc == n - 1)
            face_jac_tile<T, N, NX, NPC>(tb, L, axis, side, xa0, xa1, sa0, sa1, pm, gc, vol, wa, nu, out, pacc);
        }
      }
    }
    // ---- deterministic accumulation of time node a in the (now free) state buffer of a
    T* oa0 = ss + (a * 2) * NXY + nb;
    T* oa1 = oa0 + NXY;
    __syncthreads();                                  // every cell has read the state of a
    for (int e = tid; e < 2 * NXY; e += TL::THREADS) ss[(a * 2) * NXY + e] = 0;
    __syncthreads();
#pragma unroll 1
    for (int ph = 0; ph < 4; ++ph) {
      if (on && ((lcx & 1) | ((lcy & 1) << 1)) == ph) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < N; ++i) (c ? oa1 : oa0)[i + NX * j] += out[c][j * N + i];
      }
      __syncthreads();
    }
    // owned nodes of the tile (not on the low halo line; the last node line of the mesh
    // included), one warp per tile row
    for (int row = warp; row < 2 * NY; row += NW) {
      const int c = row / NY, iy = row - c * NY;
      const int gy = Y0 + iy;
      if (!(iy >= N - 1 && gy < N1 && (iy < NY - 1 || gy == N1 - 1))) continue;
      const T* src = ss + (a * 2 + c) * NXY + iy * NX;
      const int64_t gb = (int64_t)a * L.Nv + (int64_t)c * L.nnodes + (int64_t)gy * N1 + X0;
      for (int ix = lane; ix < NX; ix += 32) {
        const int gx = X0 + ix;
        if (ix >= N - 1 && gx < N1 && (ix < NX - 1 || gx == N1 - 1)) {
          const T v = src[ix];
          A.y[gb + ix] = rhs ? rhs[gb + ix] - v : v;
        }
      }
    }
    // the pressure rows of the owned cells
    if (on && lcx >= 1 && lcy >= 1) {
#pragma unroll
      for (int m = 0; m < NPC; ++m) {
        const int64_t gi = poff + (int64_t)a * L.Np + cell * NPC + m;
        A.y[gi] = rhs ? rhs[gi] - pacc[m] : pacc[m];
      }
    }
  }
}

// Launch of the tiled apply for an N-node, KP1-time-node level.  Returns cudaErrorNotSupported
// for configurations it does not cover (the caller then uses the colour-split kernels).
template <typename T, int N, int KP1>
cudaError_t launch_apply2d_tile(const OpArgs<T>& A, const Tab<T>& tb, const T* rhs, int n, cudaStream_t s,
                                int columns = 1) {
  using TL = Tile2D<N>;
  const size_t smem = (size_t)2 * KP1 * 2 * TL::NXY * sizeof(T);
  cudaError_t e = allow_smem(k_apply2d_tile<T, N, KP1>, smem);
  if (e != cudaSuccess) return e;
  const int tx = (n + TL::CX - 2) / (TL::CX - 1), ty = (n + TL::CY - 2) / (TL::CY - 1);
  k_apply2d_tile<T, N, KP1><<<dim3((unsigned)(tx * ty), columns), TL::THREADS, smem, s>>>(A, tb, rhs, tx);
  return cudaGetLastError();
}

}  // namespace stmg
