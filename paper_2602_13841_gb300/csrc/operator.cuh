// Matrix-free slab operator kernels: Jacobian apply y = J_n(U) x and residual R_n(U; V_prev).
//
// Sec. 4.4 ("matrix-free application of the slab Jacobian"): for every temporal basis index a
// the state-dependent spatial operator is evaluated cell-wise by sum factorisation, and the
// temporal matrices mix the results densely:
//   Y_v^i = sum_a K_ia M_h V^a + w_i [nu A_h + H'(V^i) + N^c'(V^i) + N^{b,r}] V^i + w_i (B+G^p)^T P^i
//   Y_p^i = w_i (B + G^p) V^i
// The mixing is done at the quadrature points (values sum_b K_ib JxW v^b), so each cell is
// integrated once per output time node.  The residual kernel uses the same data path with
// the nonlinear terms (Eq. InAlgNS): convective flux -v (x) v, body force w_i f(t_i), the jump
// term -phi_i(t_{n-1}^+) M_h v_{n-1} and the Nitsche data g.
//
// Kernel layout: one thread group of Q = N^D threads per cell (thread t <-> quadrature point
// t and, for the nodal stages, local node t; N = r+2 = n_q), CPB cells per block.  Cells are
// processed in 2^D colours (parity of the cell coordinates) so that cells of one launch
// share no velocity node: the scatter is race free and deterministic without atomics.
// Sum factorisation: values at the Gauss points by D one-dimensional passes with B, gradients
// by the collocation derivative Dc at the Gauss points, integration by the transposed passes.
#pragma once
#include "common.cuh"

namespace stmg {

template <int D, int N>
struct Shape {
  static constexpr int Q = (D == 2) ? N * N : N * N * N;
  static constexpr int NF = (D == 2) ? N : N * N;    // points on one face
};

// Apply the 1D matrix M (rows = output index) along dimension m to ncomp arrays of size Q
// stored contiguously in `src`, writing `dst`.  Thread t computes point t.
template <typename T, int D, int N, bool TRANSPOSE>
__device__ inline void pass_dim(const T* src, T* dst, const T (*M)[MAXN], int m, int t, int ncomp) {
  constexpr int Q = Shape<D, N>::Q;
  int stride = (m == 0) ? 1 : (m == 1 ? N : N * N);
  int im = (t / stride) % N;
  int base = t - im * stride;
  for (int c = 0; c < ncomp; ++c) {
    const T* s = src + c * Q + base;
    T acc = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) acc += (TRANSPOSE ? M[j][im] : M[im][j]) * s[j * stride];
    dst[c * Q + t] = acc;
  }
}

// Full tensor pass (all D dimensions) in place in buf, using tmp; ends with a __syncthreads.
template <typename T, int D, int N, bool TRANSPOSE>
__device__ inline void tensor_pass(T* buf, T* tmp, const T (*M)[MAXN], int t, int ncomp, bool on) {
  constexpr int Q = Shape<D, N>::Q;
  for (int m = 0; m < D; ++m) {
    const T* s = (m % 2 == 0) ? buf : tmp;
    T* d = (m % 2 == 0) ? tmp : buf;
    if (on) pass_dim<T, D, N, TRANSPOSE>(s, d, M, m, t, ncomp);
    __syncthreads();
  }
  if (D % 2 == 1) {
    if (on)
      for (int c = 0; c < ncomp; ++c) buf[c * Q + t] = tmp[c * Q + t];
    __syncthreads();
  }
}

template <typename T>
struct OpArgs {
  LevelArgs<T> L;
  const T* x;        // operand (J: increment; R: the iterate U)
  const T* state;    // J: the Newton state U (velocity part read); R: unused
  const T* vprev;    // R: V_{n-1}
  T* y;              // output (accumulated)
  int64_t xs, ys;    // batch strides (blockIdx.y selects the column of a batched apply)
  const T* geo;      // 2D: per cell [5][Q] inverse Jacobian G[0][0], G[0][1], G[1][0], G[1][1] and
                     // JxW at the quadrature points (precomputed at set-up), or null
  int64_t ss;        // batch stride of the state (0: one state shared by the batch)
  const T* nub;      // per-batch-column viscosity (device, blockIdx.y), or null: L.nu
};

// Viscosity of the batch column of this block.
template <typename T>
__device__ __forceinline__ T column_nu(const OpArgs<T>& A) { return A.nub ? A.nub[blockIdx.y] : A.L.nu; }

// The reference tables are kernel parameters; indexing them with lane-dependent indices (a
// quadrature point, a node) serialises the constant-bank reads, so the 3D kernels copy them to
// shared memory first and read them from there.
template <typename T>
__device__ __forceinline__ const Tab<T>& stage_tab(const Tab<T>& tb_param, unsigned char* s_raw) {
  static_assert(sizeof(Tab<T>) % 4 == 0, "Tab is copied in 4-byte words");
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&tb_param);
  uint32_t* dst = reinterpret_cast<uint32_t*>(s_raw);
  for (int w = threadIdx.x; w < (int)(sizeof(Tab<T>) / 4); w += blockDim.x) dst[w] = src[w];
  __syncthreads();
  return *reinterpret_cast<const Tab<T>*>(s_raw);
}

template <int D>
__device__ inline int64_t global_node(int N1, const int* cc, int r1, int t, int N) {
  int64_t g = 0, stride = 1;
  for (int l = 0; l < D; ++l) {
    int il = (l == 0) ? t % N : (l == 1 ? (t / N) % N : t / (N * N));
    g += (int64_t)(cc[l] * r1 + il) * stride;
    stride *= N1;
  }
  return g;
}

template <typename T, int D>
__device__ inline void load_corners(const LevelArgs<T>& L, const int* cc, T (*corner)[3], int t) {
  if (t < (1 << D) * D) {
    int c = t / D, i = t % D;
    int64_t v = 0, s = 1;
    for (int l = 0; l < D; ++l) { v += (int64_t)(cc[l] + ((c >> l) & 1)) * s; s *= (L.n + 1); }
    corner[c][i] = L.verts[v * D + i];
  }
}

// ---------------------------------------------------------------------------- volume kernel
enum { MJ = 0, MR = 1, MM = 2 };   // Jacobian apply, residual, mass (w_a M_h, w_a M_p)

template <typename T, int D, int N, int MODE>
__global__ void k_volume(OpArgs<T> A, Tab<T> tb_p, ColorInfo ci, int cpb) {
  __shared__ __align__(16) unsigned char s_tab[sizeof(Tab<T>)];
  const Tab<T>& tb = stage_tab(tb_p, s_tab);
  constexpr bool RES = (MODE == MR);
  constexpr bool MASS = (MODE == MM);
  constexpr int Q = Shape<D, N>::Q;
  const int kp1 = tb.k + 1, npc = tb.npc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int g = threadIdx.x / Q, t = threadIdx.x % Q;
  const int per = (MODE == MJ ? 3 : 2) * kp1 * D * Q + D * D * Q + 2 * D * Q + Q + kp1 * MAXNP + 8 * 3;
  T* s_val = sm + g * per;                        // [kp1][D][Q] increment values at qp
  T* s_tmp = s_val + kp1 * D * Q;                 // [kp1][D][Q]
  T* s_st = s_tmp + kp1 * D * Q;                  // [kp1][D][Q] state values (J only)
  T* s_F = s_st + (MODE == MJ ? kp1 * D * Q : 0);  // [D][D][Q] reference fluxes
  T* s_z = s_F + D * D * Q;                       // [D][Q] value integrand
  T* s_z2 = s_z + D * Q;                          // [D][Q] temp for the integration passes
  T* s_sp = s_z2 + D * Q;                         // [Q] pressure integrand
  T* s_pm = s_sp + Q;                             // [kp1][MAXNP] pressure modes
  T(*corner)[3] = reinterpret_cast<T(*)[3]>(s_pm + kp1 * MAXNP);

  const int cidx = blockIdx.x * cpb + g;
  const bool on = (g < cpb) && (cidx < ci.count);
  A.x += blockIdx.y * A.xs;
  A.y += blockIdx.y * A.ys;
  if (A.state) A.state += blockIdx.y * A.ss;
  const T nu = column_nu(A);
  int cc[3] = {0, 0, 0};
  if (on) decode_color_cell<D>(ci, cidx, cc);
  const LevelArgs<T>& L = A.L;
  const int r1 = N - 1;
  const int64_t gnode = on ? global_node<D>(L.N1, cc, r1, t, N) : 0;
  const int64_t cell = on ? (D == 2 ? (int64_t)cc[0] + (int64_t)L.n * cc[1]
                                    : (int64_t)cc[0] + (int64_t)L.n * (cc[1] + (int64_t)L.n * cc[2])) : 0;
  const int64_t poff = (int64_t)kp1 * L.Nv;

  if (on) {
    load_corners<T, D>(L, cc, corner, t);
    for (int b = 0; b < kp1; ++b)
      for (int c = 0; c < D; ++c) {
        int64_t gi = (int64_t)b * L.Nv + c * L.nnodes + gnode;
        s_val[(b * D + c) * Q + t] = A.x[gi];
        if (MODE == MJ) s_st[(b * D + c) * Q + t] = A.state[gi];
      }
    if (t < npc)
      for (int b = 0; b < kp1; ++b) s_pm[b * MAXNP + t] = A.x[poff + (int64_t)b * L.Np + cell * npc + t];
  }
  // the output entries of lane t (node t, pressure mode t; no other block of this colour writes
  // them): read with the inputs, so that each time node's update is a plain store
  T yo[MAXKP1][3], po[MAXKP1];
#pragma unroll
  for (int a = 0; a < MAXKP1; ++a) {
    po[a] = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) yo[a][c] = 0;
    if (on && a < kp1) {
#pragma unroll
      for (int c = 0; c < D; ++c) yo[a][c] = A.y[(int64_t)a * L.Nv + c * L.nnodes + gnode];
      if (t < npc) po[a] = A.y[poff + (int64_t)a * L.Np + cell * npc + t];
    }
  }
  __syncthreads();
  tensor_pass<T, D, N, false>(s_val, s_tmp, tb.B, t, kp1 * D, on);
  if (MODE == MJ) tensor_pass<T, D, N, false>(s_st, s_tmp, tb.B, t, kp1 * D, on);

  // geometry at quadrature point t
  int tq[3];
  tq[0] = t % N; tq[1] = (t / N) % N; tq[2] = (D == 3) ? t / (N * N) : 0;
  T G[3][3], JxW = 0, xq[3];
  T vprev_q[3] = {0, 0, 0};
  if (on) {
    T xh[3], J[3][3];
    for (int l = 0; l < D; ++l) xh[l] = tb.qx[tq[l]];
    map_jacobian<T, D>(corner, xh, J, xq);
    T det = invert<T, D>(J, G);
    JxW = det;
    for (int l = 0; l < D; ++l) JxW *= tb.qw[tq[l]];
  }
  if (RES) {
    // V_{n-1} at the quadrature points (reuse s_tmp slot 0)
    if (on)
      for (int c = 0; c < D; ++c) s_tmp[c * Q + t] = A.vprev[c * L.nnodes + gnode];
    __syncthreads();
    tensor_pass<T, D, N, false>(s_tmp, s_z2, tb.B, t, D, on);
    if (on)
      for (int c = 0; c < D; ++c) vprev_q[c] = s_tmp[c * Q + t];
    __syncthreads();
  }

  for (int a = 0; a < kp1; ++a) {
    if (on) {
      const T* va = s_val + a * D * Q;
      T gref[3][3];
      for (int c = 0; c < D; ++c)
        for (int m = 0; m < D; ++m) {
          int stride = (m == 0) ? 1 : (m == 1 ? N : N * N);
          int base = t - tq[m] * stride;
          T acc = 0;
#pragma unroll
          for (int p = 0; p < N; ++p) acc += tb.Dc[tq[m]][p] * va[c * Q + base + p * stride];
          gref[c][m] = acc;
        }
      T gp[3][3];
      for (int c = 0; c < D; ++c)
        for (int l = 0; l < D; ++l) {
          T acc = 0;
          for (int m = 0; m < D; ++m) acc += G[m][l] * gref[c][m];
          gp[c][l] = acc;
        }
      T pq = 0;
      for (int mo = 0; mo < npc; ++mo) {
        T psi = tb.P1[tq[0]][tb.modes[mo][0]] * tb.P1[tq[1]][tb.modes[mo][1]];
        if (D == 3) psi *= tb.P1[tq[2]][tb.modes[mo][2]];
        pq += psi * s_pm[a * MAXNP + mo];
      }
      T dv[3], v[3];
      for (int c = 0; c < D; ++c) {
        dv[c] = va[c * Q + t];
        v[c] = (MODE == MJ) ? s_st[(a * D + c) * Q + t] : dv[c];
      }
      const T wa = tb.w[a];
      T F[3][3];
      for (int c = 0; c < D; ++c)
        for (int l = 0; l < D; ++l) {
          T conv = RES ? v[c] * v[l] : dv[c] * v[l] + v[c] * dv[l];
          F[c][l] = MASS ? (T)0 : nu * gp[c][l] - conv - ((c == l) ? pq : (T)0);
        }
      for (int c = 0; c < D; ++c)
        for (int m = 0; m < D; ++m) {
          T acc = 0;
          for (int l = 0; l < D; ++l) acc += G[m][l] * F[c][l];
          s_F[(c * D + m) * Q + t] = wa * JxW * acc;
        }
      T fq[3] = {0, 0, 0};
      if (RES) {
        double xd[3], fd[3];
        for (int l = 0; l < D; ++l) xd[l] = (double)xq[l];
        const double ta = (double)L.t0 + 0.5 * (double)L.tau * ((double)tb.that[a] + 1.0);  // t_n^a
        if (L.problem == kProblemUser) {
          const int64_t ncells = (int64_t)ipow(L.n, D);
          for (int c = 0; c < D; ++c) fd[c] = L.ftab[(((int64_t)a * ncells + cell) * D + c) * Q + t];
        } else {
          problem_f<D>(L.problem, xd, ta, (double)L.nu, fd);
        }
        for (int c = 0; c < D; ++c) fq[c] = (T)fd[c];
      }
      for (int c = 0; c < D; ++c) {
        T acc = 0;
        if (MASS) {
          acc = wa * dv[c];
        } else {
          for (int b = 0; b < kp1; ++b) acc += tb.K[a][b] * s_val[(b * D + c) * Q + t];
        }
        if (RES) acc -= tb.C[a] * vprev_q[c] + wa * fq[c];
        s_z[c * Q + t] = JxW * acc;
      }
      T div = 0;
      for (int c = 0; c < D; ++c) div += gp[c][c];
      s_sp[t] = MASS ? wa * JxW * pq : -wa * JxW * div;
    }
    __syncthreads();
    // z_c += sum_m Dc_m^T F_cm (gradient test functions at the Gauss points)
    if (on)
      for (int c = 0; c < D; ++c) {
        T acc = s_z[c * Q + t];
        for (int m = 0; m < D; ++m) {
          int stride = (m == 0) ? 1 : (m == 1 ? N : N * N);
          int base = t - tq[m] * stride;
#pragma unroll
          for (int p = 0; p < N; ++p) acc += tb.Dc[p][tq[m]] * s_F[(c * D + m) * Q + base + p * stride];
        }
        s_z2[c * Q + t] = acc;
      }
    __syncthreads();
    tensor_pass<T, D, N, true>(s_z2, s_z, tb.B, t, D, on);
    if (on) {
      T ya[3] = {0, 0, 0}, pa = 0;
#pragma unroll
      for (int q = 0; q < MAXKP1; ++q)
        if (q == a) {
          pa = po[q];
#pragma unroll
          for (int c = 0; c < 3; ++c) ya[c] = yo[q][c];
        }
      for (int c = 0; c < D; ++c) A.y[(int64_t)a * L.Nv + c * L.nnodes + gnode] = ya[c] + s_z2[c * Q + t];
      if (t < npc) {
        T acc = 0;
        for (int q = 0; q < Q; ++q) {
          int q0 = q % N, q1 = (q / N) % N, q2 = (D == 3) ? q / (N * N) : 0;
          T psi = tb.P1[q0][tb.modes[t][0]] * tb.P1[q1][tb.modes[t][1]];
          if (D == 3) psi *= tb.P1[q2][tb.modes[t][2]];
          acc += psi * s_sp[q];
        }
        A.y[poff + (int64_t)a * L.Np + cell * npc + t] = pa + acc;
      }
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------- boundary faces
// Nitsche and boundary-convection terms on the faces of boundary cells (Eq. def-a-gam-tp,
// def-b-gam, bttp; Appendix A, Eq. DefNitscheSpatial1/10).  One thread group per boundary
// cell of one colour; the group loops over the cell's boundary faces and the time nodes, so
// no two threads of a launch touch the same velocity node.  At face point p (weight JxW_f):
//   J: a_c = w_a[-nu d_n dv_c + nu g1/h dv_c + g2/h (dv.n) n_c + dp n_c
//               + (y+ - 2y-) dv_c + (3 - sgn y)/2 (dv.n) v_c],  b_c = -w_a nu dv_c,  s = w_a dv.n
//   R: a_c = w_a[-nu d_n v_c + nu g1/h e_c + g2/h (e.n) n_c + p n_c + (y+ - 2y-) v_c + (g.n)- g_c],
//      b_c = -w_a nu e_c,  s = w_a e.n,  e = v - g
// with y = v.n, tested as  a_c z_c + b_c d_n z_c  and  s q.  h = |K| / |F| * hscale (hscale = 1/(p(p+1)) on the finest level, see LevelArgs).
template <typename T, int D, int N>
__device__ inline void face_weights(const Tab<T>& tb, int axis, int side, const int* pq, int j,
                                    T& val, T* grad) {
  int jm[3];
  jm[0] = j % N; jm[1] = (j / N) % N; jm[2] = (D == 3) ? j / (N * N) : 0;
  // tangential coordinates: dimensions other than `axis` in increasing order
  int qq[3] = {0, 0, 0};
  { int ti = 0; for (int l = 0; l < D; ++l) if (l != axis) qq[l] = pq[ti++]; }
  const bool onf = (jm[axis] == side * (N - 1));
  val = 1;
  for (int m = 0; m < D; ++m) grad[m] = 1;
  for (int l = 0; l < D; ++l) {
    T v = (l == axis) ? (onf ? (T)1 : (T)0) : tb.B[qq[l]][jm[l]];
    T dv = (l == axis) ? tb.Dend[side][jm[l]] : tb.D[qq[l]][jm[l]];
    val *= v;
    for (int m = 0; m < D; ++m) grad[m] *= (m == l) ? dv : v;
  }
}

template <typename T, int D, int N>
__device__ inline T face_psi(const Tab<T>& tb, int axis, int side, const int* pq, int mo) {
  int qq[3] = {0, 0, 0};
  { int ti = 0; for (int l = 0; l < D; ++l) if (l != axis) qq[l] = pq[ti++]; }
  T psi = 1;
  for (int l = 0; l < D; ++l)
    psi *= (l == axis) ? tb.Pend[side][tb.modes[mo][l]] : tb.P1[qq[l]][tb.modes[mo][l]];
  return psi;
}

template <typename T, int D, int N, int MODE>
__global__ void k_faces(OpArgs<T> A, Tab<T> tb_p, const int* __restrict__ bcells, int nb, int cpb) {
  __shared__ __align__(16) unsigned char s_tab[sizeof(Tab<T>)];
  const Tab<T>& tb = stage_tab(tb_p, s_tab);
  constexpr int Q = Shape<D, N>::Q;
  constexpr int NF = Shape<D, N>::NF;
  const int kp1 = tb.k + 1, npc = tb.npc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int g = threadIdx.x / Q, t = threadIdx.x % Q;
  const int per = 2 * kp1 * D * Q + kp1 * MAXNP + D * NF + D * D * NF + NF + Q + 4 + 8 * 3;
  T* s_u = sm + g * per;                 // [kp1][D][Q] operand nodal values
  T* s_st = s_u + kp1 * D * Q;           // [kp1][D][Q] state nodal values
  T* s_pm = s_st + kp1 * D * Q;          // [kp1][MAXNP]
  T* s_a = s_pm + kp1 * MAXNP;           // [D][NF]
  T* s_bg = s_a + D * NF;                // [D][D][NF]
  T* s_s = s_bg + D * D * NF;            // [NF]
  T* s_red = s_s + NF;                   // [Q]
  T* s_sc = s_red + Q;                   // [4]: volume, area
  T(*corner)[3] = reinterpret_cast<T(*)[3]>(s_sc + 4);

  constexpr bool RES = (MODE == MR);
  // with cpb == 1 each block serves one time node a0 of one cell (the time nodes' face terms are
  // independent and write different parts of y); with cpb > 1 a block loops over all time nodes
  const int a_lo = cpb == 1 ? (int)(blockIdx.x % kp1) : 0, a_hi = cpb == 1 ? a_lo + 1 : kp1;
  const int bi = cpb == 1 ? (int)(blockIdx.x / kp1) : blockIdx.x * cpb + g;
  const bool on = (g < cpb) && (bi < nb);
  const LevelArgs<T>& L = A.L;
  A.x += blockIdx.y * A.xs;
  A.y += blockIdx.y * A.ys;
  if (A.state) A.state += blockIdx.y * A.ss;
  const T nu = column_nu(A);
  int cc[3] = {0, 0, 0};
  int64_t cell = 0;
  if (on) {
    cell = bcells[bi];
    int64_t c = cell;
    for (int l = 0; l < D; ++l) { cc[l] = (int)(c % L.n); c /= L.n; }
  }
  const int64_t gnode = on ? global_node<D>(L.N1, cc, N - 1, t, N) : 0;
  const int64_t poff = (int64_t)kp1 * L.Nv;
  if (on) {
    load_corners<T, D>(L, cc, corner, t);
    for (int b = a_lo; b < a_hi; ++b)
      for (int c = 0; c < D; ++c) {
        int64_t gi = (int64_t)b * L.Nv + c * L.nnodes + gnode;
        s_u[(b * D + c) * Q + t] = A.x[gi];
        s_st[(b * D + c) * Q + t] = RES ? A.x[gi] : A.state[gi];
      }
    if (t < npc)
      for (int b = a_lo; b < a_hi; ++b) s_pm[b * MAXNP + t] = A.x[poff + (int64_t)b * L.Np + cell * npc + t];
  }
  __syncthreads();
  // cell volume |K|
  if (on) {
    int tq[3] = {t % N, (t / N) % N, (D == 3) ? t / (N * N) : 0};
    T xh[3], J[3][3], G[3][3], x[3];
    for (int l = 0; l < D; ++l) xh[l] = tb.qx[tq[l]];
    map_jacobian<T, D>(corner, xh, J, x);
    T det = invert<T, D>(J, G);
    for (int l = 0; l < D; ++l) det *= tb.qw[tq[l]];
    s_red[t] = det;
  }
  __syncthreads();
  if (on && t == 0) { T v = 0; for (int q = 0; q < Q; ++q) v += s_red[q]; s_sc[0] = v; }
  __syncthreads();

  // the faces of a cell add to the same entries of y (lane t: node t, pressure mode t): sum them
  // in registers and update y once after the face loop
  T ysum[MAXKP1][3], psum[MAXKP1];
#pragma unroll
  for (int a = 0; a < MAXKP1; ++a) { psum[a] = 0; for (int c = 0; c < 3; ++c) ysum[a][c] = 0; }
  for (int axis = 0; axis < D; ++axis)
    for (int side = 0; side < 2; ++side) {
      // uniform across the block: every group runs the loop; groups whose cell does not have
      // this boundary face stay idle (flag `has`)
      const bool has = on && (side == 0 ? cc[axis] == 0 : cc[axis] == L.n - 1);
      if (!__syncthreads_or(has)) continue;            // no cell of the block has this face
      int pq[2] = {t % N, t / N};
      T nrm[3] = {0, 0, 0}, ghat[3] = {0, 0, 0}, G[3][3], JxWf = 0, xf[3] = {0, 0, 0};
      if (has && t < NF) {
        T xh[3], J[3][3];
        { int ti = 0; for (int l = 0; l < D; ++l) xh[l] = (l == axis) ? (T)side : tb.qx[pq[ti++]]; }
        map_jacobian<T, D>(corner, xh, J, xf);
        T det = invert<T, D>(J, G);
        const T nh = side ? (T)1 : (T)-1;
        T cof[3], len2 = 0;
        for (int i = 0; i < D; ++i) { cof[i] = det * G[axis][i] * nh; len2 += cof[i] * cof[i]; }
        T dS = sqrt(len2);
        for (int i = 0; i < D; ++i) nrm[i] = cof[i] / dS;
        JxWf = dS;
        { int ti = 0; for (int l = 0; l < D; ++l) if (l != axis) JxWf *= tb.qw[pq[ti++]]; }
        for (int m = 0; m < D; ++m) { T acc = 0; for (int l = 0; l < D; ++l) acc += G[m][l] * nrm[l]; ghat[m] = acc; }
        s_red[t] = JxWf;
      }
      __syncthreads();
      if (has && t == 0) { T v = 0; for (int p = 0; p < NF; ++p) v += s_red[p]; s_sc[1] = v; }
      __syncthreads();
      const T h = has ? s_sc[0] / s_sc[1] * L.hscale : (T)1;
      for (int a = a_lo; a < a_hi; ++a) {
        if (has && t < NF) {
          T dv[3] = {0, 0, 0}, v[3] = {0, 0, 0}, gref[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
          constexpr int NN = Shape<D, N>::Q;
          for (int j = 0; j < NN; ++j) {
            T wv, wg[3];
            face_weights<T, D, N>(tb, axis, side, pq, j, wv, wg);
            for (int c = 0; c < D; ++c) {
              T u = s_u[(a * D + c) * Q + j];
              dv[c] += wv * u;
              v[c] += wv * s_st[(a * D + c) * Q + j];
              for (int m = 0; m < D; ++m) gref[c][m] += wg[m] * u;
            }
          }
          T dp = 0;
          for (int mo = 0; mo < npc; ++mo) dp += face_psi<T, D, N>(tb, axis, side, pq, mo) * s_pm[a * MAXNP + mo];
          T dn[3];
          for (int c = 0; c < D; ++c) {
            T acc = 0;
            for (int l = 0; l < D; ++l) {
              T gl = 0;
              for (int m = 0; m < D; ++m) gl += G[m][l] * gref[c][m];
              acc += gl * nrm[l];
            }
            dn[c] = acc;
          }
          T y = 0;
          for (int c = 0; c < D; ++c) y += v[c] * nrm[c];
          const T ypos = (T)0.5 * (fabs(y) + y), yneg = (T)0.5 * (fabs(y) - y);
          T e[3], gd[3] = {0, 0, 0};
          if (RES) {
            double xd[3], gv[3];
            for (int l = 0; l < D; ++l) xd[l] = (double)xf[l];
            const double ta = (double)L.t0 + 0.5 * (double)L.tau * ((double)tb.that[a] + 1.0);
            if (L.problem == kProblemUser) {
              const int64_t nf = (int64_t)ipow(L.n, D - 1), f = face_index<D>(cc, axis, L.n);
              for (int c = 0; c < D; ++c)
                gv[c] = L.gtab[(((((int64_t)a * D + axis) * 2 + side) * nf + f) * D + c) * NF + t];
            } else {
              problem_g<D>(L.problem, xd, ta, (double)L.nu, gv);
            }
            for (int c = 0; c < D; ++c) { gd[c] = (T)gv[c]; e[c] = v[c] - gd[c]; }
          } else {
            for (int c = 0; c < D; ++c) e[c] = dv[c];
          }
          T en = 0, gn = 0;
          for (int c = 0; c < D; ++c) { en += e[c] * nrm[c]; gn += gd[c] * nrm[c]; }
          const T wJ = tb.w[a] * JxWf;
          const T sgn = (y > 0) ? (T)1 : ((y < 0) ? (T)-1 : (T)0);
          for (int c = 0; c < D; ++c) {
            T ac = -nu * dn[c] + nu * L.gamma1 / h * e[c] + L.gamma2 / h * en * nrm[c] + dp * nrm[c];
            if (L.bconv) {
              if (RES) ac += (ypos - 2 * yneg) * v[c] + (T)0.5 * (fabs(gn) - gn) * gd[c];
              else ac += (ypos - 2 * yneg) * dv[c] + (T)0.5 * ((T)3 - sgn) * en * v[c];
            }
            s_a[c * NF + t] = wJ * ac;
            const T bc = -wJ * nu * e[c];
            for (int m = 0; m < D; ++m) s_bg[(c * D + m) * NF + t] = bc * ghat[m];
          }
          s_s[t] = wJ * en;
        }
        __syncthreads();
        if (has) {
          T out[3] = {0, 0, 0};
          for (int p = 0; p < NF; ++p) {
            int pp[2] = {p % N, p / N};
            T wv, wg[3];
            face_weights<T, D, N>(tb, axis, side, pp, t, wv, wg);
            for (int c = 0; c < D; ++c) {
              T acc = s_a[c * NF + p] * wv;
              for (int m = 0; m < D; ++m) acc += s_bg[(c * D + m) * NF + p] * wg[m];
              out[c] += acc;
            }
          }
#pragma unroll
          for (int q = 0; q < MAXKP1; ++q)
            if (q == a)
              for (int c = 0; c < D; ++c) ysum[q][c] += out[c];
          if (t < npc) {
            T acc = 0;
            for (int p = 0; p < NF; ++p) {
              int pp[2] = {p % N, p / N};
              acc += s_s[p] * face_psi<T, D, N>(tb, axis, side, pp, t);
            }
#pragma unroll
            for (int q = 0; q < MAXKP1; ++q)
              if (q == a) psum[q] += acc;
          }
        }
        __syncthreads();
      }
    }
  if (on) {
#pragma unroll
    for (int a = 0; a < MAXKP1; ++a) {
      if (a < a_lo || a >= a_hi) continue;
      for (int c = 0; c < D; ++c) A.y[(int64_t)a * L.Nv + c * L.nnodes + gnode] += ysum[a][c];
      if (t < npc) A.y[poff + (int64_t)a * L.Np + cell * npc + t] += psum[a];
    }
  }
}

}  // namespace stmg
