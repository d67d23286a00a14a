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
  T* EA;                // [cells][mv][mv]   element matrices of the cells ebase, ebase+1, ...
  T* EB;                // [cells][npc][mv]  (the build runs in chunks of cell planes that share
  T* EM;                // [cells][nl][nl]    one scratch; cell c is stored at c - ebase)
  int64_t ebase;
  // Patch inverse of a cell, time-diagonalised: one spatial inverse T_e^{-1} (size m_s = mv +
  // npc) per eigen-block e, column-major with stride inv_stride(m_s, element size); a complex block
  // stores (re, im) pairs.  k+1 units of m_s x stride reals per cell, storage in T, or
  T* inv;
  __half* invh;         // the same scaled to [-1, 1] in FP16 with one FP32 factor per block
  float* scale;         // [cells][nblk]
  int* status;          // set to 1 on a zero pivot
  T* work;              // global workspace of k_patch_global (null for on-chip patches) ...
  int64_t wslot;        // ... entries per block slot
};

// Column stride of a stored patch inverse: the smallest st >= m for which one m x st block of
// `es`-byte entries is a whole number of 16-byte units, so that every block and every cell's blob
// starts 16-byte aligned (the bulk copy's requirement) with the least padding (FP32, m = 38: 38).
__host__ __device__ constexpr inline int inv_stride(int m, int es) {
  int st = m;
  while (((long long)m * st * es) % 16 != 0) ++st;
  return st;
}

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
// Element matrices of one cell, computed by the whole block.  `sm` holds the per-cell tables
// (shared memory, or for cells whose tables exceed it a per-block slot of global memory).
template <typename T, int D, int N>
__device__ void elem_cell(const VankaArgs<T>& V, const Tab<T>& tb, int64_t cell, T* sm) {
  constexpr int Q = Shape<D, N>::Q;
  constexpr int NL = Q;                  // local nodes per component (N = n_q)
  constexpr int NF = Shape<D, N>::NF;
  constexpr int MV = D * NL;
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
  T* EA = V.EA + (cell - V.ebase) * (int64_t)MV * MV;
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
  T* EB = V.EB + (cell - V.ebase) * (int64_t)npc * MV;
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
  T* EM = V.EM + (cell - V.ebase) * (int64_t)NL * NL;
  for (int ent = tid; ent < NL * NL; ent += nt) {
    const int i = ent / NL, j = ent % NL;
    T acc = 0;
    for (int q = 0; q < Q; ++q) acc += s_jxw[q] * s_phi[q * NL + i] * s_phi[q * NL + j];
    EM[ent] = acc;
  }
}

// Entries of the per-cell tables of elem_cell.
template <int D, int N>
__host__ __device__ constexpr size_t elem_table_entries() {
  return (size_t)Shape<D, N>::Q * Shape<D, N>::Q * D + (size_t)Shape<D, N>::Q * Shape<D, N>::Q + Shape<D, N>::Q +
         (size_t)Shape<D, N>::Q * D + (size_t)D * Shape<D, N>::Q +
         (size_t)D * (Shape<D, N>::NF * (2 + 2 * D) + 2 * (size_t)Shape<D, N>::NF * Shape<D, N>::Q) + 8 + 24;
}

template <typename T, int D, int N>
__global__ void k_elem(VankaArgs<T> V, Tab<T> tb, int64_t c0, int64_t c1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t cell = c0 + blockIdx.x;
  if (cell >= c1) return;
  elem_cell<T, D, N>(V, tb, cell, reinterpret_cast<T*>(smem_raw));
}

// Cells whose tables exceed shared memory (3D Q4/P3): the tables live in a per-block slot of the
// global workspace V.work (elem_table_entries entries per slot); blocks stride over the cells.
template <typename T, int D, int N>
__global__ void k_elem_global(VankaArgs<T> V, Tab<T> tb, int64_t c0, int64_t c1) {
  T* sm = V.work + (int64_t)blockIdx.x * (int64_t)elem_table_entries<D, N>();
  for (int64_t cell = c0 + blockIdx.x; cell < c1; cell += gridDim.x) {
    elem_cell<T, D, N>(V, tb, cell, sm);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------- Gauss-Jordan
constexpr int kGjBatch = 8;                        // rows loaded ahead in an elimination pass
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
    // elimination: thread owns column j and every `rs`-th row (no division in the loop); rows
    // in batches of kGjBatch loads before their stores, so that a matrix in global memory is
    // not updated one dependent round trip at a time
    if (nt >= m) {
      const int rs = nt / m;
      if (tid < rs * m) {
        const int j = tid % m, chunk = tid / m;
        const T prow = S[p * ld + j];
        for (int i0 = chunk; i0 < m; i0 += kGjBatch * rs) {
          T v[kGjBatch];
#pragma unroll
          for (int u = 0; u < kGjBatch; ++u) {
            const int i = i0 + u * rs;
            v[u] = i < m ? S[i * ld + j] : (T)0;
          }
#pragma unroll
          for (int u = 0; u < kGjBatch; ++u) {
            const int i = i0 + u * rs;
            if (i < m && i != p) S[i * ld + j] = v[u] - colbuf[i] * prow;
          }
        }
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

// In-place inverse of the complex m x m matrix (Sr + i Si) (row-major, leading dimension m) by
// Gauss-Jordan elimination with partial pivoting on |a|; same structure as gauss_jordan.
template <typename T>
__device__ bool gauss_jordan_c(T* Sr, T* Si, int m, int* piv_row, T* cr, T* ci) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_pivc;
  __shared__ bool s_okc;
  if (tid == 0) s_okc = true;
  for (int p = 0; p < m; ++p) {
    if (tid < 32) {
      T best = -1; int bi = p;
      for (int i = p + tid; i < m; i += 32) {
        const T a = Sr[i * m + p] * Sr[i * m + p] + Si[i * m + p] * Si[i * m + p];
        if (a > best) { best = a; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        T ob = __shfl_down_sync(0xffffffffu, best, off);
        int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) { s_pivc = bi; piv_row[p] = bi; if (!(best > 0)) s_okc = false; }
    }
    __syncthreads();
    if (!s_okc) return false;
    const int r = s_pivc;
    if (r != p)
      for (int j = tid; j < m; j += nt) {
        T t = Sr[p * m + j]; Sr[p * m + j] = Sr[r * m + j]; Sr[r * m + j] = t;
        t = Si[p * m + j]; Si[p * m + j] = Si[r * m + j]; Si[r * m + j] = t;
      }
    __syncthreads();
    const T pr = Sr[p * m + p], pi = Si[p * m + p];
    const T den = (T)1 / (pr * pr + pi * pi);
    const T qr = pr * den, qi = -pi * den;          // 1 / (pr + i pi)
    __syncthreads();
    for (int j = tid; j < m; j += nt) {
      if (j == p) { Sr[p * m + j] = qr; Si[p * m + j] = qi; }
      else {
        const T ar = Sr[p * m + j], ai = Si[p * m + j];
        Sr[p * m + j] = ar * qr - ai * qi; Si[p * m + j] = ar * qi + ai * qr;
      }
    }
    for (int i = tid; i < m; i += nt) {
      cr[i] = (i == p) ? (T)0 : Sr[i * m + p];
      ci[i] = (i == p) ? (T)0 : Si[i * m + p];
    }
    __syncthreads();
    for (int i = tid; i < m; i += nt) if (i != p) { Sr[i * m + p] = 0; Si[i * m + p] = 0; }
    __syncthreads();
    if (nt >= m) {
      const int rs = nt / m;
      if (tid < rs * m) {
        const int j = tid % m, chunk = tid / m;
        const T br = Sr[p * m + j], bim = Si[p * m + j];
        for (int i0 = chunk; i0 < m; i0 += kGjBatch * rs) {
          T vr[kGjBatch], vi[kGjBatch];
#pragma unroll
          for (int u = 0; u < kGjBatch; ++u) {
            const int i = i0 + u * rs;
            vr[u] = i < m ? Sr[i * m + j] : (T)0;
            vi[u] = i < m ? Si[i * m + j] : (T)0;
          }
#pragma unroll
          for (int u = 0; u < kGjBatch; ++u) {
            const int i = i0 + u * rs;
            if (i < m && i != p) {
              Sr[i * m + j] = vr[u] - (cr[i] * br - ci[i] * bim);
              Si[i * m + j] = vi[u] - (cr[i] * bim + ci[i] * br);
            }
          }
        }
      }
    } else {
      for (int j = tid; j < m; j += nt) {
        const T br = Sr[p * m + j], bim = Si[p * m + j];
        for (int i = 0; i < m; ++i)
          if (i != p) {
            Sr[i * m + j] -= cr[i] * br - ci[i] * bim;
            Si[i * m + j] -= cr[i] * bim + ci[i] * br;
          }
      }
    }
    __syncthreads();
  }
  for (int p = m - 1; p >= 0; --p) {
    const int r = piv_row[p];
    if (r != p)
      for (int i = tid; i < m; i += nt) {
        T t = Sr[i * m + p]; Sr[i * m + p] = Sr[i * m + r]; Sr[i * m + r] = t;
        t = Si[i * m + p]; Si[i * m + p] = Si[i * m + r]; Si[i * m + r] = t;
      }
    __syncthreads();
  }
  return true;
}

// ---------------------------------------------------------------------------- patch build
// The cells K' around the cell at cc (offsets o in {-1, 0, 1}^D) that contain both nodes i and j
// of the cell (multi-indices im, jm within it), visited in the order of the offset code
// nb = (o0 + 1) + 3 (o1 + 1) + 9 (o2 + 1): f(nc, ii, jj) gets K''s linear index and the two nodes'
// local indices in K'.  Per dimension at most two offsets qualify (0, and -1 or +1 when both
// nodes lie on that side), so a patch entry visits 1 to 2^D cells instead of testing 3^D.
template <int D, int N, typename F>
__device__ __forceinline__ void for_shared_cells(const int* cc, int n, const int* im, const int* jm, F&& f) {
  int off[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  int cnt[3] = {1, 1, 1};
  for (int l = 0; l < D; ++l) {
    cnt[l] = 0;
    for (int o = -1; o <= 1; ++o) {
      const int x = cc[l] + o, a = im[l] - o * (N - 1), b = jm[l] - o * (N - 1);
      if (x >= 0 && x < n && a >= 0 && a < N && b >= 0 && b < N) off[l][cnt[l]++] = o;
    }
  }
  for (int u2 = 0; u2 < cnt[2]; ++u2)
    for (int u1 = 0; u1 < cnt[1]; ++u1)
      for (int u0 = 0; u0 < cnt[0]; ++u0) {
        const int o[3] = {off[0][u0], off[1][u1], off[2][u2]};
        int64_t nc = 0, s = 1;
        int ii = 0, jj = 0, si = 1;
        for (int l = 0; l < D; ++l) {
          nc += (int64_t)(cc[l] + o[l]) * s;
          s *= n;
          ii += (im[l] - o[l] * (N - 1)) * si;
          jj += (jm[l] - o[l] * (N - 1)) * si;
          si *= N;
        }
        f(nc, ii, jj);
      }
}

// Spatial patch ordering: velocity (c, i) -> c*NL + i, then pressure mode m -> MV + m.  The
// surrogate patch matrix of Eq. vanka0 is, time node by time node,
//   S~ = [ K^tau (x) M + W (x) A ,  W (x) B^T ;  W (x) B , 0 ],   W = diag(w_a),
// with the cell's assembled velocity mass M (per component), velocity block A (viscous,
// convection at v*, Nitsche) and divergence block B.  With W^{-1} K^tau = Q diag(lam) Q^{-1}
// it is similar to the block diagonal of T_lam = [lam M + A, B^T; B, 0]: one spatial inverse
// per eigenvalue instead of one inverse of the whole space-time patch (Sec. 4.3).
template <typename T, int D, int N>
__device__ bool patch_cell(const VankaArgs<T>& V, const Tab<T>& tb, const TEig<T>& te, int64_t cell, T* Sr, T* Si,
                           T* Ap, T* Mp, T* cr, T* ci, int* piv) {
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int npc = tb.npc, kp1 = tb.k + 1;
  const int ms = MV + npc, st = inv_stride(ms, V.invh ? 2 : (int)sizeof(T));
  const LevelArgs<T>& L = V.L;
  int cc[3] = {0, 0, 0};
  cell_coords<D>(cell, L.n, cc);
  const int tid = threadIdx.x, nt = blockDim.x;
  // assembled velocity and mass blocks: sum over neighbours K' sharing both nodes
  for (int ent = tid; ent < MV * MV; ent += nt) {
    const int row = ent / MV, col = ent % MV;
    const int c = row / NL, i = row % NL, e = col / NL, j = col % NL;
    int im[3], jm[3];
    node_multi<D, N>(i, im); node_multi<D, N>(j, jm);
    T acc = 0;
    for_shared_cells<D, N>(cc, L.n, im, jm, [&](int64_t nc, int ii, int jj) {
      acc += V.EA[(nc - V.ebase) * (int64_t)MV * MV + (int64_t)(c * NL + ii) * MV + e * NL + jj];
    });
    Ap[ent] = acc;
  }
  for (int ent = tid; ent < NL * NL; ent += nt) {
    const int i = ent / NL, j = ent % NL;
    int im[3], jm[3];
    node_multi<D, N>(i, im); node_multi<D, N>(j, jm);
    T acc = 0;
    for_shared_cells<D, N>(cc, L.n, im, jm, [&](int64_t nc, int ii, int jj) {
      acc += V.EM[(nc - V.ebase) * (int64_t)NL * NL + (int64_t)ii * NL + jj];
    });
    Mp[ent] = acc;
  }
  __syncthreads();
  const T* EB = V.EB + (cell - V.ebase) * (int64_t)npc * MV;
  const int64_t cbase = cell * (int64_t)kp1 * ms * st;
  for (int e = 0; e < te.nblk; ++e) {
    const bool cplx = te.cplx[e] != 0;
    const T lr = te.lre[e], li = te.lim[e];
    for (int ent = tid; ent < ms * ms; ent += nt) {
      const int row = ent / ms, col = ent % ms;
      T vr = 0, vi = 0;
      if (row < MV && col < MV) {
        vr = Ap[row * MV + col];
        if (row / NL == col / NL) {
          const T mm = Mp[(row % NL) * NL + (col % NL)];
          vr += lr * mm; vi = li * mm;
        }
      } else if (row < MV) {
        vr = EB[(col - MV) * MV + row];
      } else if (col < MV) {
        vr = EB[(row - MV) * MV + col];
      }
      Sr[ent] = vr;
      Si[ent] = vi;
    }
    __syncthreads();
    const bool ok = cplx ? gauss_jordan_c<T>(Sr, Si, ms, piv, cr, ci) : gauss_jordan<T>(Sr, ms, ms, piv, cr);
    if (!ok) { if (tid == 0) *V.status = 1; return false; }
    const int w = cplx ? 2 : 1;                                  // reals per stored entry
    const int64_t bbase = cbase + (int64_t)te.off[e] * ms * st;  // in reals
    if (V.invh) {
      T mx = 0;
      for (int ent = tid; ent < ms * ms; ent += nt) mx = fmax(mx, fmax(fabs(Sr[ent]), cplx ? fabs(Si[ent]) : (T)0));
      mx = block_absmax<T>(mx);
      // the scale is held in FP32: divide by exactly the value the apply multiplies by
      const float sc = mx > 0 ? (float)mx : 1.f;
      const T isc = (T)1 / (T)sc;
      if (tid == 0) V.scale[cell * te.nblk + e] = sc;
      __half* inv = V.invh + bbase;
      for (int ent = tid; ent < ms * st; ent += nt) {
        const int j = ent / st, i = ent % st;
        const bool in = i < ms;
        inv[(int64_t)w * ent] = __float2half_rn(in ? (float)(Sr[i * ms + j] * isc) : 0.f);
        if (cplx) inv[(int64_t)w * ent + 1] = __float2half_rn(in ? (float)(Si[i * ms + j] * isc) : 0.f);
      }
    } else {
      T* inv = V.inv + bbase;
      for (int ent = tid; ent < ms * st; ent += nt) {
        const int j = ent / st, i = ent % st;     // column-major: inv[j][i] = T^{-1}[i][j]
        const bool in = i < ms;                   // rows ms..st-1 pad the column
        inv[(int64_t)w * ent] = in ? Sr[i * ms + j] : (T)0;
        if (cplx) inv[(int64_t)w * ent + 1] = in ? Si[i * ms + j] : (T)0;
      }
    }
    __syncthreads();
  }
  return true;
}

// Patches whose matrices fit shared memory: one block per cell.
template <typename T, int D, int N>
__global__ void k_patch(VankaArgs<T> V, Tab<T> tb, TEig<T> te, int64_t c0, int64_t c1) {
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int ms = MV + tb.npc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Sr = reinterpret_cast<T*>(smem_raw);           // [ms][ms]
  T* Si = Sr + ms * ms;                             // [ms][ms] imaginary part
  T* Ap = Si + ms * ms;                             // [MV][MV] assembled velocity block
  T* Mp = Ap + MV * MV;                             // [NL][NL] assembled scalar mass
  T* cr = Mp + NL * NL;                             // [ms]
  T* ci = cr + ms;                                  // [ms]
  int* piv = reinterpret_cast<int*>(ci + ms);       // [ms]
  const int64_t cell = c0 + blockIdx.x;
  if (cell >= c1) return;
  patch_cell<T, D, N>(V, tb, te, cell, Sr, Si, Ap, Mp, cr, ci, piv);
}

// Larger patches (3D, r >= 2): the matrices live in a per-block slot of a global workspace
// (V.work, V.wslot entries per slot; the slots together stay L2-resident); blocks stride over
// the cells.  Only the pivot bookkeeping is in shared memory.
template <typename T, int D, int N>
__global__ void __launch_bounds__(512, 2) k_patch_global(VankaArgs<T> V, Tab<T> tb, TEig<T> te, int64_t c0, int64_t c1) {
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int ms = MV + tb.npc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* cr = reinterpret_cast<T*>(smem_raw);           // [ms]
  T* ci = cr + ms;                                  // [ms]
  int* piv = reinterpret_cast<int*>(ci + ms);       // [ms]
  T* Sr = V.work + (int64_t)blockIdx.x * V.wslot;
  T* Si = Sr + ms * ms;
  T* Ap = Si + ms * ms;
  T* Mp = Ap + MV * MV;
  for (int64_t cell = c0 + blockIdx.x; cell < c1; cell += gridDim.x) {
    if (!patch_cell<T, D, N>(V, tb, te, cell, Sr, Si, Ap, Mp, cr, ci, piv)) return;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------- sweep
// d[patch] += W~ S~^{-1} res[patch] for the cells of one colour (W~ = omega on velocity,
// omega_p on pressure DoFs), through the time-diagonalised inverse (k_patch):
//   rt_e = sum_a F[e][a] res_a  (per spatial patch DoF),  yhat_e = T_e^{-1} rt_e,
//   y_a = sum_e Re(G[a][e] yhat_e).
// One block per cell.  Its inverse ((k+1) m_s x stride reals, contiguous) is staged into shared
// memory by one bulk asynchronous copy (cp.async.bulk, completion on an mbarrier) issued before
// the residual gather, so the whole blob is in flight while the block gathers and transforms
// the residual; thread i then owns spatial row i of every block.  Accumulation in T.

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(bar), "r"(phase) : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for phase `phase` of the mbarrier: gives up after `limit_ns` of wall time (and in
// any case after 2^26 rounds).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase, uint64_t limit_ns) {
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 63) == 63 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}
constexpr int kBulkChunk = 32768;                // bytes per bulk copy instruction
constexpr uint64_t kWaitLimit = 1000000000ull;   // 1 s before the wait is declared failed

template <typename SI> struct InvLd;
template <> struct InvLd<float> {
  __device__ static float re(const float* p) { return *p; }
  __device__ static float2 cx(const float* p) { return *reinterpret_cast<const float2*>(p); }
};
template <> struct InvLd<double> {
  __device__ static double re(const double* p) { return *p; }
  __device__ static double2 cx(const double* p) { return *reinterpret_cast<const double2*>(p); }
};
template <> struct InvLd<__half> {
  __device__ static float re(const __half* p) { return __half2float(*p); }
  __device__ static float2 cx(const __half* p) { return __half22float2(*reinterpret_cast<const __half2*>(p)); }
};

// Rows of the spatial Vanka patch of Q_{N-1} / P_{N-2}^disc: D N^D velocity DoFs and C(r+D, D)
// pressure modes (r = N - 2), known at compile time so that the row products unroll.
template <int D, int N>
__host__ __device__ constexpr int patch_rows() {
  return D * Shape<D, N>::Q + (D == 2 ? (N - 1) * N / 2 : (N - 1) * N * (N + 1) / 6);
}

// Dynamic shared memory of k_vanka_apply: [blob | rt (kp1 x mr T) | gb (ms int64) | mbarrier].
__host__ __device__ inline size_t apply_blob_bytes(int kp1, int ms, size_t si) {
  return ((size_t)kp1 * ms * inv_stride(ms, (int)si) * si + 127) & ~(size_t)127;
}
__host__ __device__ inline size_t apply_smem_bytes(int kp1, int ms, size_t si, size_t t) {
  const int mr = (ms + 1) & ~1;
  return apply_blob_bytes(kp1, ms, si) + (((size_t)kp1 * mr * t + 7) & ~(size_t)7) + (size_t)ms * 8 + 16;
}
// One cell's slot of a multi-cell block, rounded so that every slot's blob starts 128-byte aligned.
__host__ __device__ inline size_t apply_slot_bytes(int kp1, int ms, size_t si, size_t t) {
  return (apply_smem_bytes(kp1, ms, si, t) + 127) & ~(size_t)127;
}

// Slot strides of a batched sweep (blockIdx.y = slot): inverse entries, FP16 scales, vector entries.
struct SlotStrides { int64_t inv, scale, vec; };

template <typename T, typename SI, int D, int N>
__global__ void k_vanka_apply(LevelArgs<T> L, const SI* __restrict__ inv, const float* __restrict__ scale,
                              const T* __restrict__ res, T* __restrict__ d, T omega, T omega_p, int kp1, int npc,
                              TEig<T> te, ColorInfo ci, int* __restrict__ wstat, unsigned extra_tx,
                              SlotStrides zs) {
  inv += blockIdx.y * zs.inv;
  if (scale) scale += blockIdx.y * zs.scale;
  res += blockIdx.y * zs.vec;
  d += blockIdx.y * zs.vec;
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int ms = MV + npc, st = inv_stride(ms, (int)sizeof(SI)), mr = (ms + 1) & ~1;
  // small patches: several cells per block (slots of tpc threads), so that more cells are in
  // flight than the 32-blocks-per-SM limit would allow with one-warp blocks
  const int tpc = ((ms + 31) / 32) * 32, slot = threadIdx.x / tpc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + (size_t)slot * apply_slot_bytes(kp1, ms, sizeof(SI), sizeof(T));
  const size_t blob = apply_blob_bytes(kp1, ms, sizeof(SI));
  SI* sinv = reinterpret_cast<SI*>(base);
  T* rt = reinterpret_cast<T*>(base + blob);                                          // [kp1 units][mr]
  int64_t* gb = reinterpret_cast<int64_t*>(base + blob + (((size_t)kp1 * mr * sizeof(T) + 7) & ~(size_t)7));
  uint64_t* bar = reinterpret_cast<uint64_t*>(gb + ms);
  const int cidx = blockIdx.x * (blockDim.x / tpc) + slot;
  const bool active = cidx < ci.count;
  const int tid = threadIdx.x - slot * tpc, nt = tpc;
  int cc[3] = {0, 0, 0};
  int64_t cell = 0;
  if (active) {
    decode_color_cell<D>(ci, cidx, cc);
    int64_t s = 1;
    for (int l = 0; l < D; ++l) { cell += (int64_t)cc[l] * s; s *= L.n; }
  }
  // stage the cell's inverse: one thread per slot arms the barrier and issues the bulk copies
  const uint32_t b = smem_addr(bar);
  const uint32_t bytes = (uint32_t)((size_t)kp1 * ms * st * sizeof(SI));
  if (active && tid == 0) {
    mbar_init(b, 1);
    mbar_expect_tx(b, bytes + extra_tx);            // extra_tx > 0 only under the failure-test hook
    const unsigned char* src = reinterpret_cast<const unsigned char*>(inv + cell * (int64_t)kp1 * ms * st);
    for (uint32_t o = 0; o < bytes; o += kBulkChunk) {
      const uint32_t n = bytes - o < (uint32_t)kBulkChunk ? bytes - o : (uint32_t)kBulkChunk;
      bulk_g2s(smem_addr(base + o), src + o, n, b);
    }
  }
  // meanwhile: gather the residual on the patch and transform it to the time eigenbasis; each
  // thread also reads the current correction on its own row (no other block of this colour
  // touches these entries), so the update at the end is a plain store
  T dold[MAXKP1];
#pragma unroll
  for (int a = 0; a < MAXKP1; ++a) dold[a] = 0;
  for (int l = tid; active && l < ms; l += nt) {
    int64_t g, sa;
    if (l < MV) {
      const int c = l / NL, i = l % NL;
      g = c * L.nnodes + global_node<D>(L.N1, cc, N - 1, i, N);
      sa = L.Nv;
    } else {
      g = (int64_t)kp1 * L.Nv + cell * npc + (l - MV);
      sa = L.Np;
    }
    gb[l] = g;
    T ra[MAXKP1];
#pragma unroll
    for (int a = 0; a < MAXKP1; ++a) ra[a] = a < kp1 ? res[g + a * sa] : (T)0;
    if (l == tid) {
#pragma unroll
      for (int a = 0; a < MAXKP1; ++a) dold[a] = a < kp1 ? d[g + a * sa] : (T)0;
    }
    for (int e = 0; e < te.nblk; ++e) {
      T fr = 0, fi = 0;
#pragma unroll
      for (int a = 0; a < MAXKP1; ++a) { fr += te.Fre[e][a] * ra[a]; fi += te.Fim[e][a] * ra[a]; }
      rt[te.off[e] * mr + l] = fr;
      if (te.cplx[e]) rt[(te.off[e] + 1) * mr + l] = fi;
    }
  }
  __syncthreads();                                   // barriers initialised, rt and gb complete
  if (!active) return;
  if (!mbar_wait_bounded(b, 0, kWaitLimit)) {
    // the copy did not complete in time: report, give it a second bounded wait (it writes this
    // slot's shared memory) and leave d unchanged for this cell
    if (tid == 0) atomicExch(wstat, 1);
    mbar_wait_bounded(b, 0, kWaitLimit);
    return;
  }
  const int i = tid;
  if (i >= ms) return;
  T yr[MAXKP1], yi[MAXKP1];
#pragma unroll
  for (int e = 0; e < MAXKP1; ++e) { yr[e] = 0; yi[e] = 0; }
  for (int e = 0; e < te.nblk; ++e) {
    const SI* blk = sinv + (int64_t)te.off[e] * ms * st;
    const T* r0 = rt + te.off[e] * mr;
    T ar = 0, ai = 0;
    if (!te.cplx[e]) {
      for (int j = 0; j < ms; ++j) ar += (T)InvLd<SI>::re(blk + j * st + i) * r0[j];
    } else {
      const T* r1 = r0 + mr;
      for (int j = 0; j < ms; ++j) {
        const auto v = InvLd<SI>::cx(blk + 2 * (j * st + i));
        const T vr = (T)v.x, vi = (T)v.y, xr = r0[j], xi = r1[j];
        ar += vr * xr - vi * xi;
        ai += vr * xi + vi * xr;
      }
    }
    const T sc = scale ? (T)scale[cell * te.nblk + e] : (T)1;
#pragma unroll
    for (int q = 0; q < MAXKP1; ++q)
      if (q == e) { yr[q] = sc * ar; yi[q] = sc * ai; }
  }
  const int64_t g = gb[i];
  const int64_t sa = i < MV ? L.Nv : L.Np;
  const T wgt = i < MV ? omega : omega_p;
#pragma unroll
  for (int a = 0; a < MAXKP1; ++a) {
    if (a >= kp1) break;
    T y = 0;
#pragma unroll
    for (int e = 0; e < MAXKP1; ++e)
      if (e < te.nblk) y += te.Gre[a][e] * yr[e] - te.Gim[a][e] * yi[e];
    d[g + a * sa] = dold[a] + wgt * y;
  }
}

// Warp-specialised persistent form of k_vanka_apply for patches whose inverse is small (the 2D
// levels).  A block owns a ring of S stages in shared memory and walks the cells cidx =
// blockIdx.x + t gridDim.x (t = 0, 1, ...) of the colour.  Warp 0 produces: one lane streams the
// inverse of cell t into stage t % S by bulk copies (the stage's full barrier) as soon as the
// cell that used the stage before has been solved (its empty barrier).  C consumer groups of TPC
// threads solve the cells t = g, g + C, ...: thread i of a group owns row i, gathers the residual
// and correction of the group's next cell into registers before it waits for the current
// inverse, and the group releases the stage when it is done.  Copies thus stay in flight while
// cells are solved and C cells are solved at once, instead of every block waiting for its own
// copy, solving and ending.  Cells of one colour have disjoint patches, so a correction gathered
// ahead is still current when its cell is solved.  The products are those of k_vanka_apply, in
// the same order.
// Shared memory: [S stages | C rt buffers (kp1 x mr T) | full[S] | empty[S] | abort flag].
// rt rows of the persistent kernel are padded to a multiple of 4 entries, so that every unit row
// starts on a 16-byte boundary and is read four entries at a time.
__host__ __device__ inline int ws_rt_row(int ms) { return (ms + 3) & ~3; }
__host__ __device__ inline size_t ws_rt_bytes(int kp1, int ms, size_t t) {
  return ((size_t)kp1 * ws_rt_row(ms) * t + 15) & ~(size_t)15;
}

// Row i of the product of a stored inverse block with the vector r (real block) or with r0 + i r1
// (complex block, entries interleaved re/im), over the patch rows j = 0 .. MS - 1 in order; r, r0
// and r1 are 16-byte aligned shared-memory rows read as vectors of 16 bytes (4 floats / 2 doubles).
template <typename T, typename SI, int MS>
__device__ __forceinline__ T row_product_re(const SI* blk, int i, const T* r) {
  constexpr int W = 16 / sizeof(T);
  constexpr int st = inv_stride(MS, (int)sizeof(SI));   // compile time: immediate load offsets
  T ar = 0;
#pragma unroll
  for (int j0 = 0; j0 < MS; j0 += W) {
    T x[W];
    if constexpr (W == 4) {
      const float4 v = *reinterpret_cast<const float4*>(r + j0);
      x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
      const double2 v = *reinterpret_cast<const double2*>(r + j0);
      x[0] = v.x; x[1] = v.y;
    }
#pragma unroll
    for (int u = 0; u < W; ++u)
      if (j0 + u < MS) ar += (T)InvLd<SI>::re(blk + (j0 + u) * st + i) * x[u];
  }
  return ar;
}
template <typename T, typename SI, int MS>
__device__ __forceinline__ void row_product_cx(const SI* blk, int i, const T* r0, const T* r1, T* ar_out,
                                               T* ai_out) {
  constexpr int W = 16 / sizeof(T);
  constexpr int st = inv_stride(MS, (int)sizeof(SI));
  T ar = 0, ai = 0;
#pragma unroll
  for (int j0 = 0; j0 < MS; j0 += W) {
    T xr[W], xi[W];
    if constexpr (W == 4) {
      const float4 a = *reinterpret_cast<const float4*>(r0 + j0);
      const float4 b = *reinterpret_cast<const float4*>(r1 + j0);
      xr[0] = a.x; xr[1] = a.y; xr[2] = a.z; xr[3] = a.w;
      xi[0] = b.x; xi[1] = b.y; xi[2] = b.z; xi[3] = b.w;
    } else {
      const double2 a = *reinterpret_cast<const double2*>(r0 + j0);
      const double2 b = *reinterpret_cast<const double2*>(r1 + j0);
      xr[0] = a.x; xr[1] = a.y;
      xi[0] = b.x; xi[1] = b.y;
    }
#pragma unroll
    for (int u = 0; u < W; ++u)
      if (j0 + u < MS) {
        const auto v = InvLd<SI>::cx(blk + 2 * ((j0 + u) * st + i));
        const T vr = (T)v.x, vi = (T)v.y;
        ar += vr * xr[u] - vi * xi[u];
        ai += vr * xi[u] + vi * xr[u];
      }
  }
  *ar_out = ar;
  *ai_out = ai;
}
__host__ __device__ inline size_t ws_smem_bytes(int kp1, int ms, size_t si, size_t t, int S, int C) {
  return (size_t)S * apply_blob_bytes(kp1, ms, si) + (size_t)C * ws_rt_bytes(kp1, ms, t) + (size_t)2 * S * 8 + 16;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Named barrier `id` over n threads that also returns whether v held in all of them.
__device__ __forceinline__ bool group_and(int id, int n, bool v) {
  uint32_t r;
  asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
               : "=r"(r) : "r"((uint32_t)v), "r"(id), "r"(n) : "memory");
  return r != 0;
}
__device__ __forceinline__ void group_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Global index of patch row l of the cell at cc (velocity: component-major nodes; pressure: the
// cell's modes after the (k+1) velocity blocks) and the stride between its time nodes.
template <typename T, int D, int N>
__device__ __forceinline__ int64_t patch_row_index(const LevelArgs<T>& L, const int* cc, int64_t cell, int l,
                                                   int kp1, int npc, int64_t* sa) {
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  if (l < MV) {
    *sa = L.Nv;
    return (l / NL) * L.nnodes + global_node<D>(L.N1, cc, N - 1, l % NL, N);
  }
  *sa = L.Np;
  return (int64_t)kp1 * L.Nv + cell * npc + (l - MV);
}

template <typename T, typename SI, int D, int N>
__global__ void k_vanka_apply_ws(LevelArgs<T> L, const SI* __restrict__ inv, const float* __restrict__ scale,
                                 const T* __restrict__ res, T* __restrict__ d, T omega, T omega_p, int kp1, int npc,
                                 TEig<T> te, ColorInfo ci, int* __restrict__ wstat, unsigned extra_tx,
                                 SlotStrides zs, int S, int C, int TPC) {
  inv += blockIdx.y * zs.inv;
  if (scale) scale += blockIdx.y * zs.scale;
  res += blockIdx.y * zs.vec;
  d += blockIdx.y * zs.vec;
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int ms = MV + npc, st = inv_stride(ms, (int)sizeof(SI)), mr = ws_rt_row(ms);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t blob = apply_blob_bytes(kp1, ms, sizeof(SI));
  const size_t rtb = ws_rt_bytes(kp1, ms, sizeof(T));
  unsigned char* rt_base = smem_raw + (size_t)S * blob;
  uint64_t* full = reinterpret_cast<uint64_t*>(rt_base + (size_t)C * rtb);
  uint64_t* empty = full + S;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + S);
  const int tid = threadIdx.x;
  const int G = (int)gridDim.x;
  const int ncell = ci.count > (int)blockIdx.x ? (ci.count - (int)blockIdx.x + G - 1) / G : 0;
  if (ncell == 0) return;                                                             // block-uniform
  const uint32_t bytes = (uint32_t)((size_t)kp1 * ms * st * sizeof(SI));
  auto cell_of = [&](int t, int* cc) -> int64_t {
    decode_color_cell<D>(ci, (int)blockIdx.x + t * G, cc);
    int64_t c = 0, m = 1;
    for (int l = 0; l < D; ++l) { c += (int64_t)cc[l] * m; m *= L.n; }
    return c;
  };
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_addr(full + s), 1);
      mbar_init(smem_addr(empty + s), 1);
    }
    *abort_flag = 0;
  }
  __syncthreads();                                   // barriers initialised
  int issued = 0;                                    // producer lane: cells whose copies were issued
  if (tid < 32) {
    if (tid == 0) {
      for (int t = 0; t < ncell; ++t) {
        if (*abort_flag) break;
        const int s = t % S;
        if (t >= S) {
          // cell t - S has been solved: the stage is free
          if (!mbar_wait_bounded(smem_addr(empty + s), (uint32_t)(((t / S) - 1) & 1), kWaitLimit)) {
            atomicExch(wstat, 1);
            *abort_flag = 1;
            break;
          }
          // order the consumers' generic reads of the stage before the async-proxy writes
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        int cc[3] = {0, 0, 0};
        const int64_t c = cell_of(t, cc);
        const uint32_t b = smem_addr(full + s);
        mbar_expect_tx(b, bytes + (t == 0 ? extra_tx : 0u));   // extra_tx > 0 only under the failure-test hook
        const unsigned char* src = reinterpret_cast<const unsigned char*>(inv + c * (int64_t)kp1 * ms * st);
        unsigned char* dst = smem_raw + (size_t)s * blob;
        for (uint32_t o = 0; o < bytes; o += kBulkChunk) {
          const uint32_t n = bytes - o < (uint32_t)kBulkChunk ? bytes - o : (uint32_t)kBulkChunk;
          bulk_g2s(smem_addr(dst + o), src + o, n, b);
        }
        issued = t + 1;
      }
    }
  } else if ((tid - 32) / TPC < C) {
    const int g = (tid - 32) / TPC, i = (tid - 32) % TPC;
    T* rt = reinterpret_cast<T*>(rt_base + (size_t)g * rtb);
    const bool row = i < ms;
    int64_t gi = 0, sa = 0, cell = 0;
    T ra[MAXKP1] = {}, dold[MAXKP1] = {};
    // row i of cell t: global index, residual and old correction (registers)
    auto gather = [&](int t) {
      int cc[3] = {0, 0, 0};
      cell = cell_of(t, cc);
      if (!row) return;
      gi = patch_row_index<T, D, N>(L, cc, cell, i, kp1, npc, &sa);
#pragma unroll
      for (int a = 0; a < MAXKP1; ++a) {
        ra[a] = a < kp1 ? res[gi + a * sa] : (T)0;
        dold[a] = a < kp1 ? d[gi + a * sa] : (T)0;
      }
    };
    if (g < ncell) gather(g);
    for (int t = g; t < ncell; t += C) {
      const int s = t % S;
      // the time-eigenbasis transform of this cell's residual
      if (row) {
        for (int e = 0; e < te.nblk; ++e) {
          T fr = 0, fi = 0;
#pragma unroll
          for (int a = 0; a < MAXKP1; ++a) { fr += te.Fre[e][a] * ra[a]; fi += te.Fim[e][a] * ra[a]; }
          rt[te.off[e] * mr + i] = fr;
          if (te.cplx[e]) rt[(te.off[e] + 1) * mr + i] = fi;
        }
      }
      const int64_t gcur = gi, scur = sa, ccur = cell;
      T dcur[MAXKP1];
#pragma unroll
      for (int a = 0; a < MAXKP1; ++a) dcur[a] = dold[a];
      // the group's next cell: its gather is in flight while this one waits and is solved
      if (t + C < ncell) gather(t + C);
      bool ok = mbar_wait_bounded(smem_addr(full + s), (uint32_t)((t / S) & 1), kWaitLimit);
      ok = group_and(1 + g, TPC, ok && !*abort_flag);   // rt complete; one decision for the group
      if (!ok) {
        if (i == 0) { atomicExch(wstat, 1); *abort_flag = 1; }
        break;
      }
      if (row) {
        const SI* sinv = reinterpret_cast<const SI*>(smem_raw + (size_t)s * blob);
        T yr[MAXKP1], yi[MAXKP1];
#pragma unroll
        for (int e = 0; e < MAXKP1; ++e) { yr[e] = 0; yi[e] = 0; }
        for (int e = 0; e < te.nblk; ++e) {
          const SI* blk = sinv + (int64_t)te.off[e] * ms * st;
          const T* r0 = rt + te.off[e] * mr;
          T ar = 0, ai = 0;
          if (!te.cplx[e]) ar = row_product_re<T, SI, patch_rows<D, N>()>(blk, i, r0);
          else row_product_cx<T, SI, patch_rows<D, N>()>(blk, i, r0, r0 + mr, &ar, &ai);
          const T sc = scale ? (T)scale[ccur * te.nblk + e] : (T)1;
#pragma unroll
          for (int q = 0; q < MAXKP1; ++q)
            if (q == e) { yr[q] = sc * ar; yi[q] = sc * ai; }
        }
        const T wgt = i < MV ? omega : omega_p;
#pragma unroll
        for (int a = 0; a < MAXKP1; ++a) {
          if (a >= kp1) break;
          T y = 0;
#pragma unroll
          for (int e = 0; e < MAXKP1; ++e)
            if (e < te.nblk) y += te.Gre[a][e] * yr[e] - te.Gim[a][e] * yi[e];
          d[gcur + a * scur] = dcur[a] + wgt * y;
        }
      }
      group_sync(1 + g, TPC);                        // the group is done with stage s and rt
      if (i == 0) mbar_arrive(smem_addr(empty + s));
    }
  }
  __syncthreads();
  // after a failure, copies may still be in flight: wait (bounded) for the latest use of every
  // stage before the block's shared memory is given up
  if (tid == 0 && *abort_flag) {
    for (int s = 0; s < S && s < issued; ++s) {
      const int u = (issued - 1 - s) / S;            // latest use of stage s: cell s + u S
      mbar_wait_bounded(smem_addr(full + s), (uint32_t)(u & 1), kWaitLimit);
    }
  }
}

// Patches whose inverse blob exceeds shared memory (3D, r >= 2): the same arithmetic as
// k_vanka_apply, each thread streaming its row of every block straight from global memory.
template <typename SI> struct InvLdG;
template <> struct InvLdG<float> {
  __device__ static float re(const float* p) { return __ldg(p); }
  __device__ static float2 cx(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
};
template <> struct InvLdG<double> {
  __device__ static double re(const double* p) { return __ldg(p); }
  __device__ static double2 cx(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }
};
template <> struct InvLdG<__half> {
  __device__ static float re(const __half* p) { return __half2float(__ldg(p)); }
  __device__ static float2 cx(const __half* p) { return __half22float2(__ldg(reinterpret_cast<const __half2*>(p))); }
};

template <typename T, typename SI, int D, int N>
__global__ void k_vanka_apply_global(LevelArgs<T> L, const SI* __restrict__ inv, const float* __restrict__ scale,
                                     const T* __restrict__ res, T* __restrict__ d, T omega, T omega_p, int kp1,
                                     int npc, TEig<T> te, ColorInfo ci, SlotStrides zs) {
  inv += blockIdx.y * zs.inv;
  if (scale) scale += blockIdx.y * zs.scale;
  res += blockIdx.y * zs.vec;
  d += blockIdx.y * zs.vec;
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int ms = MV + npc, st = inv_stride(ms, (int)sizeof(SI)), mr = (ms + 1) & ~1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rt = reinterpret_cast<T*>(smem_raw);                                              // [kp1 units][mr]
  int64_t* gb = reinterpret_cast<int64_t*>(smem_raw + (((size_t)kp1 * mr * sizeof(T) + 7) & ~(size_t)7));
  const int cidx = blockIdx.x;
  if (cidx >= ci.count) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  int cc[3] = {0, 0, 0};
  decode_color_cell<D>(ci, cidx, cc);
  int64_t cell = 0, s = 1;
  for (int l = 0; l < D; ++l) { cell += (int64_t)cc[l] * s; s *= L.n; }
  // each thread also reads the current correction on its own row (no other block of this
  // colour touches these entries), so the update at the end is a plain store
  T dold[MAXKP1];
#pragma unroll
  for (int a = 0; a < MAXKP1; ++a) dold[a] = 0;
  for (int l = tid; l < ms; l += nt) {
    int64_t g, sa;
    if (l < MV) {
      const int c = l / NL, i = l % NL;
      g = c * L.nnodes + global_node<D>(L.N1, cc, N - 1, i, N);
      sa = L.Nv;
    } else {
      g = (int64_t)kp1 * L.Nv + cell * npc + (l - MV);
      sa = L.Np;
    }
    gb[l] = g;
    T ra[MAXKP1];
#pragma unroll
    for (int a = 0; a < MAXKP1; ++a) ra[a] = a < kp1 ? res[g + a * sa] : (T)0;
    if (l == tid) {
#pragma unroll
      for (int a = 0; a < MAXKP1; ++a) dold[a] = a < kp1 ? d[g + a * sa] : (T)0;
    }
    for (int e = 0; e < te.nblk; ++e) {
      T fr = 0, fi = 0;
#pragma unroll
      for (int a = 0; a < MAXKP1; ++a) { fr += te.Fre[e][a] * ra[a]; fi += te.Fim[e][a] * ra[a]; }
      rt[te.off[e] * mr + l] = fr;
      if (te.cplx[e]) rt[(te.off[e] + 1) * mr + l] = fi;
    }
  }
  __syncthreads();
  const int i = tid;
  if (i >= ms) return;
  const SI* base = inv + cell * (int64_t)kp1 * ms * st;
  T yr[MAXKP1], yi[MAXKP1];
#pragma unroll
  for (int e = 0; e < MAXKP1; ++e) { yr[e] = 0; yi[e] = 0; }
  for (int e = 0; e < te.nblk; ++e) {
    const SI* blk = base + (int64_t)te.off[e] * ms * st;
    const T* r0 = rt + te.off[e] * mr;
    T ar = 0, ai = 0;
    if (!te.cplx[e]) {
      for (int j = 0; j < ms; ++j) ar += (T)InvLdG<SI>::re(blk + (int64_t)j * st + i) * r0[j];
    } else {
      const T* r1 = r0 + mr;
      for (int j = 0; j < ms; ++j) {
        const auto v = InvLdG<SI>::cx(blk + 2 * ((int64_t)j * st + i));
        const T vr = (T)v.x, vi = (T)v.y, xr = r0[j], xi = r1[j];
        ar += vr * xr - vi * xi;
        ai += vr * xi + vi * xr;
      }
    }
    const T sc = scale ? (T)scale[cell * te.nblk + e] : (T)1;
#pragma unroll
    for (int q = 0; q < MAXKP1; ++q)
      if (q == e) { yr[q] = sc * ar; yi[q] = sc * ai; }
  }
  const int64_t g = gb[i];
  const int64_t sa = i < MV ? L.Nv : L.Np;
  const T wgt = i < MV ? omega : omega_p;
#pragma unroll
  for (int a = 0; a < MAXKP1; ++a) {
    if (a >= kp1) break;
    T y = 0;
#pragma unroll
    for (int e = 0; e < MAXKP1; ++e)
      if (e < te.nblk) y += te.Gre[a][e] * yr[e] - te.Gim[a][e] * yi[e];
    d[g + a * sa] = dold[a] + wgt * y;
  }
}

}  // namespace stmg
