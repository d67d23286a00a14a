// Inexact space-time Vanka smoother (Sec. 4.3, Eq. LVS, vanka0, DefTildeHn, DefVnAst).
//
// Build (per level, at the level state U):
//   1. v* = sum_a phi_a(t*) V^a at the slab midpoint (one spatial field);
//   2. k_elem: per cell K the spatial element matrices at v*:
//        A_K = nu A + H'(v*) + N^c'(v*) + N^{b,r}   (velocity x velocity, boundary faces included)
//        B_K = B + G^p                                (pressure x velocity)
//        M_K                                          (scalar velocity mass)
//   3. k_patch: the patch matrix is the global submatrix on the DoFs of K (all velocity and
//      pressure DoFs of K at all k+1 time nodes), so the velocity blocks sum the element
//      matrices of every neighbour cell sharing both DoFs:
//        S~_K = [ K^tau (x) M_patch + M^tau (x) A_patch ,  M^tau (x) B_K^T ]
//               [ M^tau (x) B_K                         ,  0               ]
//      M^tau = diag(w_a).  S~_K is inverted in shared memory by Gauss-Jordan elimination with
//      partial pivoting; the inverse is stored column-major per cell.
// Sweep (additive, damped): d <- d + omega sum_K R_K^T S~_K^{-1} R_K (rhs - J d); cells are
// updated in 2^d colours so that the scatter is race free and deterministic.
#pragma once
#include <cuda_fp16.h>

#include "operator.cuh"

namespace stmg {

template <typename T>
struct VankaArgs {
  LevelArgs<T> L;
  const T* vstar;       // midpoint velocity field (Nv)
  T* EA;                // [cells][mv][mv]
  T* EB;                // [cells][npc][mv]
  T* EM;                // [cells][nl][nl]
  T* inv;               // [cells][mst][mst] column-major inverse (storage in T), or
  __half* invh;         // the same scaled to [-1, 1] in FP16 with one FP32 factor per cell
  float* scale;         // [cells]
  int* status;          // set to 1 on a zero pivot
};

// Column stride of a stored patch inverse: m rounded up to 8 entries (16-byte aligned columns).
__host__ __device__ inline int inv_stride(int m) { return (m + 7) & ~7; }

// max |x| over the block (all threads receive it)
template <typename T>
__device__ inline T block_absmax(T v) {
  __shared__ T wmax[32];
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wmax[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (int)((blockDim.x + 31) >> 5)) ? wmax[lane] : (T)0;
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane == 0) wmax[0] = v;
  }
  __syncthreads();
  v = wmax[0];
  __syncthreads();
  return v;
}

template <int D>
__device__ inline void cell_coords(int64_t cell, int n, int* cc) {
  for (int l = 0; l < D; ++l) { cc[l] = (int)(cell % n); cell /= n; }
}

template <int D, int N>
__device__ inline void node_multi(int i, int* im) {
  im[0] = i % N; im[1] = (i / N) % N; im[2] = (D == 3) ? i / (N * N) : 0;
}

// ---------------------------------------------------------------------------- element matrices
template <typename T, int D, int N>
__global__ void k_elem(VankaArgs<T> V, Tab<T> tb, int64_t ncells) {
  constexpr int Q = Shape<D, N>::Q;
  constexpr int NL = Q;                  // local nodes per component (N = n_q)
  constexpr int NF = Shape<D, N>::NF;
  constexpr int MV = D * NL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* s_gphi = sm;                        // [Q][NL][D] physical basis gradients
  T* s_phi = s_gphi + Q * NL * D;        // [Q][NL]
  T* s_jxw = s_phi + Q * NL;             // [Q]
  T* s_v = s_jxw + Q;                    // [Q][D] v* at quadrature points
  T* s_vn = s_v + Q * D;                 // [D][NL] v* nodal
  T* s_f = s_vn + D * NL;                // per face: [NF] jxw, [NF][D] n, [NF] y, [NF][D] v, [NF][NL] phi, [NF][NL] dn
  constexpr int FSZ = NF * (2 + 2 * D) + 2 * NF * NL;
  T* s_misc = s_f + D * FSZ;             // [8]: volume, area
  T(*corner)[3] = reinterpret_cast<T(*)[3]>(s_misc + 8);
  __shared__ int s_faces[6];
  __shared__ int s_nf;

  const int64_t cell = blockIdx.x;
  if (cell >= ncells) return;
  const LevelArgs<T>& L = V.L;
  int cc[3] = {0, 0, 0};
  cell_coords<D>(cell, L.n, cc);
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid < (1 << D) * D) {
    int c = tid / D, i = tid % D;
    int64_t v = 0, s = 1;
    for (int l = 0; l < D; ++l) { v += (int64_t)(cc[l] + ((c >> l) & 1)) * s; s *= (L.n + 1); }
    corner[c][i] = L.verts[v * D + i];
  }
  for (int e = tid; e < D * NL; e += nt) {
    int c = e / NL, i = e % NL;
    s_vn[e] = V.vstar[c * L.nnodes + global_node<D>(L.N1, cc, N - 1, i, N)];
  }
  if (tid == 0) {
    int nf = 0;
    for (int ax = 0; ax < D; ++ax) {
      if (cc[ax] == 0) s_faces[nf++] = ax * 2 + 0;
      if (cc[ax] == L.n - 1) s_faces[nf++] = ax * 2 + 1;
    }
    s_nf = nf;
  }
  __syncthreads();
  // volume quadrature data
  for (int q = tid; q < Q; q += nt) {
    int tq[3]; node_multi<D, N>(q, tq);
    T xh[3], J[3][3], G[3][3], x[3];
    for (int l = 0; l < D; ++l) xh[l] = tb.qx[tq[l]];
    map_jacobian<T, D>(corner, xh, J, x);
    T det = invert<T, D>(J, G);
    T w = det;
    for (int l = 0; l < D; ++l) w *= tb.qw[tq[l]];
    s_jxw[q] = w;
    for (int j = 0; j < NL; ++j) {
      int jm[3]; node_multi<D, N>(j, jm);
      T val = 1, gr[3] = {1, 1, 1};
      for (int l = 0; l < D; ++l) {
        val *= tb.B[tq[l]][jm[l]];
        for (int m = 0; m < D; ++m) gr[m] *= (m == l) ? tb.D[tq[l]][jm[l]] : tb.B[tq[l]][jm[l]];
      }
      s_phi[q * NL + j] = val;
      for (int l = 0; l < D; ++l) {
        T acc = 0;
        for (int m = 0; m < D; ++m) acc += G[m][l] * gr[m];
        s_gphi[(q * NL + j) * D + l] = acc;
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < Q * D; e += nt) {
    int q = e / D, c = e % D;
    T acc = 0;
    for (int j = 0; j < NL; ++j) acc += s_phi[q * NL + j] * s_vn[c * NL + j];
    s_v[e] = acc;
  }
  if (tid == 0) { T v = 0; for (int q = 0; q < Q; ++q) v += s_jxw[q]; s_misc[0] = v; }
  __syncthreads();
  // boundary face data (one buffer per boundary face of this cell)
  const int nfaces = s_nf;
  for (int f = 0; f < nfaces; ++f) {
    const int axis = s_faces[f] / 2, side = s_faces[f] % 2;
    T* F = s_f + f * FSZ;
    T* f_jxw = F; T* f_n = F + NF; T* f_y = f_n + NF * D; T* f_v = f_y + NF; T* f_phi = f_v + NF * D;
    T* f_dn = f_phi + NF * NL;
    for (int p = tid; p < NF; p += nt) {
      int pq[2] = {p % N, p / N};
      int qq[3] = {0, 0, 0};
      { int ti = 0; for (int l = 0; l < D; ++l) if (l != axis) qq[l] = pq[ti++]; }
      T xh[3], J[3][3], G[3][3], x[3];
      for (int l = 0; l < D; ++l) xh[l] = (l == axis) ? (T)side : tb.qx[qq[l]];
      map_jacobian<T, D>(corner, xh, J, x);
      T det = invert<T, D>(J, G);
      const T nh = side ? (T)1 : (T)-1;
      T cof[3], len2 = 0;
      for (int i = 0; i < D; ++i) { cof[i] = det * G[axis][i] * nh; len2 += cof[i] * cof[i]; }
      T dS = sqrt(len2), w = dS;
      for (int l = 0; l < D; ++l) if (l != axis) w *= tb.qw[qq[l]];
      f_jxw[p] = w;
      T nrm[3];
      for (int i = 0; i < D; ++i) { nrm[i] = cof[i] / dS; f_n[p * D + i] = nrm[i]; }
      T ghat[3];
      for (int m = 0; m < D; ++m) { T acc = 0; for (int l = 0; l < D; ++l) acc += G[m][l] * nrm[l]; ghat[m] = acc; }
      T vv[3] = {0, 0, 0};
      for (int j = 0; j < NL; ++j) {
        T wv, wg[3];
        face_weights<T, D, N>(tb, axis, side, pq, j, wv, wg);
        T dn = 0;
        for (int m = 0; m < D; ++m) dn += ghat[m] * wg[m];
        f_phi[p * NL + j] = wv;
        f_dn[p * NL + j] = dn;
        for (int c = 0; c < D; ++c) vv[c] += wv * s_vn[c * NL + j];
      }
      T y = 0;
      for (int c = 0; c < D; ++c) { f_v[p * D + c] = vv[c]; y += vv[c] * nrm[c]; }
      f_y[p] = y;
    }
    __syncthreads();
    if (tid == 0) { T a = 0; for (int p = 0; p < NF; ++p) a += f_jxw[p]; s_misc[1 + f] = a; }
    __syncthreads();
  }
  // velocity block: entry (c, i ; e, j) = row (test c, i), column (trial e, j)
  T* EA = V.EA + cell * (int64_t)MV * MV;
  for (int ent = tid; ent < MV * MV; ent += nt) {
    const int row = ent / MV, col = ent % MV;
    const int c = row / NL, i = row % NL, e = col / NL, j = col % NL;
    T acc = 0;
    for (int q = 0; q < Q; ++q) {
      const T* gi = s_gphi + (q * NL + i) * D;
      const T* gj = s_gphi + (q * NL + j) * D;
      const T pj = s_phi[q * NL + j];
      T t = -s_v[q * D + c] * pj * gi[e];
      if (c == e) {
        T lap = 0, adv = 0;
        for (int l = 0; l < D; ++l) { lap += gi[l] * gj[l]; adv += s_v[q * D + l] * gi[l]; }
        t += L.nu * lap - pj * adv;
      }
      acc += s_jxw[q] * t;
    }
    for (int f = 0; f < nfaces; ++f) {
      const T* F = s_f + f * FSZ;
      const T* f_jxw = F; const T* f_n = F + NF; const T* f_y = f_n + NF * D; const T* f_v = f_y + NF;
      const T* f_phi = f_v + NF * D; const T* f_dn = f_phi + NF * NL;
      const T h = s_misc[0] / s_misc[1 + f] * L.hscale;
      for (int p = 0; p < NF; ++p) {
        const T pi = f_phi[p * NL + i], pj = f_phi[p * NL + j];
        const T y = f_y[p];
        const T ypos = (T)0.5 * (fabs(y) + y), yneg = (T)0.5 * (fabs(y) - y);
        const T sgn = (y > 0) ? (T)1 : ((y < 0) ? (T)-1 : (T)0);
        T t = L.gamma2 / h * f_n[p * D + c] * f_n[p * D + e] * pj * pi;
        if (c == e) {
          t += -L.nu * f_dn[p * NL + j] * pi - L.nu * pj * f_dn[p * NL + i] + L.nu * L.gamma1 / h * pj * pi;
          if (L.bconv) t += (ypos - 2 * yneg) * pj * pi;
        }
        if (L.bconv) t += (T)0.5 * ((T)3 - sgn) * f_n[p * D + e] * pj * f_v[p * D + c] * pi;
        acc += f_jxw[p] * t;
      }
    }
    EA[ent] = acc;
  }
  // pressure x velocity block B_K[m][(e, j)]
  const int npc = tb.npc;
  T* EB = V.EB + cell * (int64_t)npc * MV;
  for (int ent = tid; ent < npc * MV; ent += nt) {
    const int m = ent / MV, col = ent % MV, e = col / NL, j = col % NL;
    T acc = 0;
    for (int q = 0; q < Q; ++q) {
      int tq[3]; node_multi<D, N>(q, tq);
      T psi = tb.P1[tq[0]][tb.modes[m][0]] * tb.P1[tq[1]][tb.modes[m][1]];
      if (D == 3) psi *= tb.P1[tq[2]][tb.modes[m][2]];
      acc -= s_jxw[q] * psi * s_gphi[(q * NL + j) * D + e];
    }
    for (int f = 0; f < nfaces; ++f) {
      const int axis = s_faces[f] / 2, side = s_faces[f] % 2;
      const T* F = s_f + f * FSZ;
      const T* f_jxw = F; const T* f_n = F + NF; const T* f_phi = f_n + NF * D + NF + NF * D;
      for (int p = 0; p < NF; ++p) {
        int pq[2] = {p % N, p / N};
        acc += f_jxw[p] * face_psi<T, D, N>(tb, axis, side, pq, m) * f_n[p * D + e] * f_phi[p * NL + j];
      }
    }
    EB[ent] = acc;
  }
  T* EM = V.EM + cell * (int64_t)NL * NL;
  for (int ent = tid; ent < NL * NL; ent += nt) {
    const int i = ent / NL, j = ent % NL;
    T acc = 0;
    for (int q = 0; q < Q; ++q) acc += s_jxw[q] * s_phi[q * NL + i] * s_phi[q * NL + j];
    EM[ent] = acc;
  }
}

// ---------------------------------------------------------------------------- Gauss-Jordan
// In-place inverse of the m x m row-major matrix S (leading dimension ld) with partial (row)
// pivoting; column interchanges undo the row interchanges at the end.  All threads of the
// block take part; returns false (block-uniformly) on a zero pivot.
template <typename T>
__device__ bool gauss_jordan(T* S, int m, int ld, int* piv_row, T* colbuf) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_piv;
  __shared__ bool s_ok;
  if (tid == 0) s_ok = true;
  for (int p = 0; p < m; ++p) {
    if (tid < 32) {
      T best = -1; int bi = p;
      for (int i = p + tid; i < m; i += 32) {
        T a = fabs(S[i * ld + p]);
        if (a > best) { best = a; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        T ob = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) { s_piv = bi; piv_row[p] = bi; if (!(best > 0)) s_ok = false; }
    }
    __syncthreads();
    if (!s_ok) return false;
    const int r = s_piv;
    if (r != p)
      for (int j = tid; j < m; j += nt) { T t = S[p * ld + j]; S[p * ld + j] = S[r * ld + j]; S[r * ld + j] = t; }
    __syncthreads();
    const T pinv = (T)1 / S[p * ld + p];
    __syncthreads();
    for (int j = tid; j < m; j += nt) S[p * ld + j] = (j == p) ? pinv : S[p * ld + j] * pinv;
    for (int i = tid; i < m; i += nt) {
      colbuf[i] = (i == p) ? (T)0 : S[i * ld + p];
    }
    __syncthreads();
    for (int i = tid; i < m; i += nt) if (i != p) S[i * ld + p] = 0;
    __syncthreads();
    // elimination: thread owns column j and every `rs`-th row (no division in the loop)
    if (nt >= m) {
      const int rs = nt / m;
      if (tid < rs * m) {
        const int j = tid % m, chunk = tid / m;
        const T prow = S[p * ld + j];
        for (int i = chunk; i < m; i += rs)
          if (i != p) S[i * ld + j] -= colbuf[i] * prow;
      }
    } else {
      for (int j = tid; j < m; j += nt) {
        const T prow = S[p * ld + j];
        for (int i = 0; i < m; ++i)
          if (i != p) S[i * ld + j] -= colbuf[i] * prow;
      }
    }
    __syncthreads();
  }
  for (int p = m - 1; p >= 0; --p) {
    const int r = piv_row[p];
    if (r != p)
      for (int i = tid; i < m; i += nt) { T t = S[i * ld + p]; S[i * ld + p] = S[i * ld + r]; S[i * ld + r] = t; }
    __syncthreads();
  }
  return true;
}

// ---------------------------------------------------------------------------- patch build
// Patch-local ordering: velocity (a, c, i) -> a*MV + c*NL + i, then pressure (a, m) ->
// KP1*MV + a*npc + m.
template <typename T, int D, int N>
__global__ void k_patch(VankaArgs<T> V, Tab<T> tb, int64_t ncells) {
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int kp1 = tb.k + 1, npc = tb.npc;
  const int m = kp1 * (MV + npc);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);           // [m][m]
  T* Ap = S + m * m;                                // [MV][MV] assembled velocity block
  T* Mp = Ap + MV * MV;                             // [NL][NL] assembled scalar mass
  T* colbuf = Mp + NL * NL;                         // [m]
  int* piv = reinterpret_cast<int*>(colbuf + m);    // [m]
  const int64_t cell = blockIdx.x;
  if (cell >= ncells) return;
  const LevelArgs<T>& L = V.L;
  int cc[3] = {0, 0, 0};
  cell_coords<D>(cell, L.n, cc);
  const int tid = threadIdx.x, nt = blockDim.x;
  constexpr int NNB = (D == 2) ? 9 : 27;
  // assembled velocity and mass blocks: sum over neighbours K' sharing both nodes
  for (int ent = tid; ent < MV * MV; ent += nt) {
    const int row = ent / MV, col = ent % MV;
    const int c = row / NL, i = row % NL, e = col / NL, j = col % NL;
    int im[3], jm[3];
    node_multi<D, N>(i, im); node_multi<D, N>(j, jm);
    T acc = 0;
    for (int nb = 0; nb < NNB; ++nb) {
      int o[3] = {nb % 3 - 1, (nb / 3) % 3 - 1, nb / 9 - 1};
      bool ok = true;
      int64_t nc = 0, s = 1;
      int ii = 0, jj = 0, si = 1;
      for (int l = 0; l < D; ++l) {
        int x = cc[l] + o[l];
        int a = im[l] - o[l] * (N - 1), b = jm[l] - o[l] * (N - 1);
        if (x < 0 || x >= L.n || a < 0 || a >= N || b < 0 || b >= N) { ok = false; break; }
        nc += (int64_t)x * s; s *= L.n;
        ii += a * si; jj += b * si; si *= N;
      }
      if (ok) acc += V.EA[nc * (int64_t)MV * MV + (int64_t)(c * NL + ii) * MV + e * NL + jj];
    }
    Ap[ent] = acc;
  }
  for (int ent = tid; ent < NL * NL; ent += nt) {
    const int i = ent / NL, j = ent % NL;
    int im[3], jm[3];
    node_multi<D, N>(i, im); node_multi<D, N>(j, jm);
    T acc = 0;
    for (int nb = 0; nb < NNB; ++nb) {
      int o[3] = {nb % 3 - 1, (nb / 3) % 3 - 1, nb / 9 - 1};
      bool ok = true;
      int64_t nc = 0, s = 1;
      int ii = 0, jj = 0, si = 1;
      for (int l = 0; l < D; ++l) {
        int x = cc[l] + o[l];
        int a = im[l] - o[l] * (N - 1), b = jm[l] - o[l] * (N - 1);
        if (x < 0 || x >= L.n || a < 0 || a >= N || b < 0 || b >= N) { ok = false; break; }
        nc += (int64_t)x * s; s *= L.n;
        ii += a * si; jj += b * si; si *= N;
      }
      if (ok) acc += V.EM[nc * (int64_t)NL * NL + (int64_t)ii * NL + jj];
    }
    Mp[ent] = acc;
  }
  __syncthreads();
  const T* EB = V.EB + cell * (int64_t)npc * MV;
  for (int ent = tid; ent < m * m; ent += nt) {
    const int row = ent / m, col = ent % m;
    T v = 0;
    if (row < kp1 * MV && col < kp1 * MV) {
      const int a = row / MV, rv = row % MV, b = col / MV, cv = col % MV;
      if (rv / NL == cv / NL) v = tb.K[a][b] * Mp[(rv % NL) * NL + (cv % NL)];
      if (a == b) v += tb.w[a] * Ap[rv * MV + cv];
    } else if (row < kp1 * MV) {
      const int a = row / MV, rv = row % MV, b = (col - kp1 * MV) / npc, pm = (col - kp1 * MV) % npc;
      if (a == b) v = tb.w[a] * EB[pm * MV + rv];
    } else if (col < kp1 * MV) {
      const int a = (row - kp1 * MV) / npc, pm = (row - kp1 * MV) % npc, b = col / MV, cv = col % MV;
      if (a == b) v = tb.w[a] * EB[pm * MV + cv];
    }
    S[ent] = v;
  }
  __syncthreads();
  bool ok = gauss_jordan<T>(S, m, m, piv, colbuf);
  if (!ok) { if (tid == 0) *V.status = 1; return; }
  if (V.invh) {
    T mx = 0;
    for (int ent = tid; ent < m * m; ent += nt) mx = fmax(mx, fabs(S[ent]));
    mx = block_absmax<T>(mx);
    // the scale is held in FP32: divide by exactly the value the apply multiplies by
    const float sc = mx > 0 ? (float)mx : 1.f;
    const T isc = (T)1 / (T)sc;
    if (tid == 0) V.scale[cell] = sc;
    const int ms = inv_stride(m);
    __half* inv = V.invh + cell * (int64_t)m * ms;
    for (int ent = tid; ent < m * ms; ent += nt) {
      const int j = ent / ms, i = ent % ms;
      inv[ent] = __float2half_rn(i < m ? (float)(S[i * m + j] * isc) : 0.f);
    }
    return;
  }
  const int ms = inv_stride(m);
  T* inv = V.inv + cell * (int64_t)m * ms;
  for (int ent = tid; ent < m * ms; ent += nt) {
    const int j = ent / ms, i = ent % ms;        // column-major store: inv[j][i] = S^{-1}[i][j]
    inv[ent] = i < m ? S[i * m + j] : (T)0;      // rows m..ms-1 pad the column to 16 bytes
  }
}

// ---------------------------------------------------------------------------- sweep
// d[patch] += omega * S~^{-1} res[patch] for the cells of one colour.
//
// The inverse of a patch is stored column-major with a padded column stride ms = inv_stride(m)
// in SI = T, or in FP16 scaled per cell by scale[cell].  TPC threads (a multiple of 32) serve
// one cell and a block holds blockDim / TPC cells.  A thread owns RR consecutive rows (1 for T,
// 2 for FP16: one 4-byte load per column either way, so FP16 halves the bytes at the same
// instruction count) and keeps kApplyUnroll column loads in flight before their FMAs; the
// threads of a cell read each column as one contiguous segment.  Accumulation in T.
constexpr int kApplyUnroll = 8;

template <typename SI> struct InvRows;
template <> struct InvRows<float> {
  static constexpr int RR = 1;
  using raw = float;
  __device__ static raw ld(const float* p) { return __ldg(p); }
  __device__ static void get(raw v, float* o) { o[0] = v; }
};
template <> struct InvRows<double> {
  static constexpr int RR = 1;
  using raw = double;
  __device__ static raw ld(const double* p) { return __ldg(p); }
  __device__ static void get(raw v, double* o) { o[0] = v; }
};
template <> struct InvRows<__half> {
  static constexpr int RR = 2;
  using raw = __half2;
  __device__ static raw ld(const __half* p) { return __ldg(reinterpret_cast<const __half2*>(p)); }
  __device__ static void get(raw v, float* o) { const float2 f = __half22float2(v); o[0] = f.x; o[1] = f.y; }
};
template <typename SI> struct InvVal { using type = SI; };
template <> struct InvVal<__half> { using type = float; };

template <typename T, typename SI, int D, int N>
__global__ void k_vanka_apply(LevelArgs<T> L, const SI* __restrict__ inv, const float* __restrict__ scale,
                              const T* __restrict__ res, T* __restrict__ d, T omega, T omega_p, int kp1, int npc,
                              int tpc, ColorInfo ci) {
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  constexpr int RR = InvRows<SI>::RR;
  using V = typename InvVal<SI>::type;
  using W = typename InvRows<SI>::raw;
  const int m = kp1 * (MV + npc), ms = inv_stride(m), mr = (m + 1) & ~1;
  const int cpb = blockDim.x / tpc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = threadIdx.x / tpc, tid = threadIdx.x % tpc;
  T* r = reinterpret_cast<T*>(smem_raw) + slot * mr;
  int64_t* gidx = reinterpret_cast<int64_t*>(reinterpret_cast<T*>(smem_raw) + cpb * mr) + slot * m;
  const int cidx = blockIdx.x * cpb + slot;
  const bool active = cidx < ci.count;
  int64_t cell = 0;
  if (active) {
    int cc[3] = {0, 0, 0};
    decode_color_cell<D>(ci, cidx, cc);
    int64_t s = 1;
    for (int l = 0; l < D; ++l) { cell += (int64_t)cc[l] * s; s *= L.n; }
    for (int l = tid; l < m; l += tpc) {
      int64_t g;
      if (l < kp1 * MV) {
        const int a = l / MV, rv = l % MV, c = rv / NL, i = rv % NL;
        g = (int64_t)a * L.Nv + c * L.nnodes + global_node<D>(L.N1, cc, N - 1, i, N);
      } else {
        const int a = (l - kp1 * MV) / npc, pm = (l - kp1 * MV) % npc;
        g = (int64_t)kp1 * L.Nv + (int64_t)a * L.Np + cell * npc + pm;
      }
      gidx[l] = g;
      r[l] = res[g];
    }
  }
  __syncthreads();
  const int i0 = tid * RR;
  if (!active || i0 >= m) return;
  const SI* col = inv + cell * (int64_t)m * ms + i0;
  T acc[RR];
#pragma unroll
  for (int t = 0; t < RR; ++t) acc[t] = 0;
  int j = 0;
  for (; j + kApplyUnroll <= m; j += kApplyUnroll) {
    W w[kApplyUnroll];
#pragma unroll
    for (int u = 0; u < kApplyUnroll; ++u) w[u] = InvRows<SI>::ld(col + (int64_t)(j + u) * ms);
#pragma unroll
    for (int u = 0; u < kApplyUnroll; ++u) {
      V v[RR];
      InvRows<SI>::get(w[u], v);
      const T ru = r[j + u];
#pragma unroll
      for (int t = 0; t < RR; ++t) acc[t] += (T)v[t] * ru;
    }
  }
  for (; j < m; ++j) {
    V v[RR];
    InvRows<SI>::get(InvRows<SI>::ld(col + (int64_t)j * ms), v);
    const T rj = r[j];
#pragma unroll
    for (int t = 0; t < RR; ++t) acc[t] += (T)v[t] * rj;
  }
  const T sc = scale ? (T)scale[cell] : (T)1;
#pragma unroll
  for (int t = 0; t < RR; ++t) {
    const int i = i0 + t;
    if (i < m) d[gidx[i]] += (i < kp1 * MV ? omega : omega_p) * sc * acc[t];
  }
}

}  // namespace stmg
