// Diagonal space-time Vanka: the cheaper smoother named as future work in the paper's closing
// section (diagonal Vanka, John 2000, carried to the space-time patch).  The velocity block of the
// surrogate patch S~_K (Eq. vanka0, DefTildeHn) keeps only the couplings of each spatial velocity
// DoF with itself -- one (k+1) x (k+1) temporal block
//     T_ci = K^tau M_ii + W A_(ci)(ci),      W = diag(w_a)
// per velocity patch DoF ci = (component c, node i), with M and A the neighbour-summed (global)
// diagonal entries -- and the pressure coupling W (x) B_K stays whole.  The modified patch
//     [A_d, (W (x) B)^T; W (x) B, 0]
// is solved exactly through its pressure Schur complement S = (W (x) B) A_d^{-1} (W (x) B)^T of
// size (k+1) npc:
//     y = A_d^{-1} r_v,  p = S^{-1} ((W (x) B) y - r_p),  v = y - A_d^{-1} (W (x) B)^T p.
// Stored per cell ("diagonal blob", precision T): T_ci^{-1} for every ci ([MV][k+1][k+1]), B_K
// ([npc][MV]) and S^{-1} ([(k+1) npc][(k+1) npc], row-major) -- e.g. 804 reals for 2D Q3/P2 DG(2)
// instead of 4332 for the time-diagonalised full patch, 3088 instead of 81608 for 3D Q3/P2 DG(1).
#pragma once
#include "vanka.cuh"

namespace stmg {

__host__ __device__ inline int64_t diag_blob_entries(int mv, int npc, int kp1) {
  return (int64_t)mv * kp1 * kp1 + (int64_t)npc * mv + (int64_t)(kp1 * npc) * (kp1 * npc);
}

// Inverse of the small dense n x n matrix A (row-major, n <= 3) into Ai by Gauss-Jordan with
// partial pivoting, in registers of one thread.  Returns false on a zero pivot.
template <typename T>
__device__ inline bool small_inverse(const T (&A)[MAXKP1][MAXKP1], int n, T (&Ai)[MAXKP1][MAXKP1]) {
  T M[MAXKP1][2 * MAXKP1];
#pragma unroll
  for (int i = 0; i < MAXKP1; ++i)
#pragma unroll
    for (int j = 0; j < 2 * MAXKP1; ++j) M[i][j] = (j < MAXKP1) ? A[i][j] : (T)(j - MAXKP1 == i ? 1 : 0);
  for (int p = 0; p < n; ++p) {
    int r = p;
    for (int i = p + 1; i < n; ++i)
      if (fabs(M[i][p]) > fabs(M[r][p])) r = i;
    if (!(fabs(M[r][p]) > (T)0)) return false;
    if (r != p)
      for (int j = 0; j < 2 * MAXKP1; ++j) { T t = M[p][j]; M[p][j] = M[r][j]; M[r][j] = t; }
    const T piv = (T)1 / M[p][p];
    for (int j = 0; j < 2 * MAXKP1; ++j) M[p][j] *= piv;
    for (int i = 0; i < n; ++i) {
      if (i == p) continue;
      const T f = M[i][p];
      for (int j = 0; j < 2 * MAXKP1; ++j) M[i][j] -= f * M[p][j];
    }
  }
#pragma unroll
  for (int i = 0; i < MAXKP1; ++i)
#pragma unroll
    for (int j = 0; j < MAXKP1; ++j) Ai[i][j] = M[i][j + MAXKP1];
  return true;
}

// One block per cell: diagonal blob of the cell from the element matrices of the cell and its
// neighbours (the scratch of k_elem).
template <typename T, int D, int N>
__global__ void k_patch_diag(VankaArgs<T> V, Tab<T> tb, int64_t c0, int64_t c1) {
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  constexpr int NNB = (D == 2) ? 9 : 27;
  const int npc = tb.npc, kp1 = tb.k + 1, ns = kp1 * npc;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_ti = reinterpret_cast<T*>(smem_raw);           // [MV][kp1][kp1] inverse temporal blocks
  T* s_S = s_ti + MV * kp1 * kp1;                     // [ns][ns] Schur complement
  int* s_piv = reinterpret_cast<int*>(s_S + ns * ns); // [ns]
  T* s_col = reinterpret_cast<T*>(s_piv + ns + (ns & 1)); // [ns]
  const int64_t cell = c0 + blockIdx.x;
  if (cell >= c1) return;
  const LevelArgs<T>& L = V.L;
  int cc[3] = {0, 0, 0};
  cell_coords<D>(cell, L.n, cc);
  const int tid = threadIdx.x, nt = blockDim.x;
  T* blob = V.inv + cell * diag_blob_entries(MV, npc, kp1);
  // temporal blocks of every velocity patch DoF: neighbour-summed diagonal of A and of M
  for (int ci = tid; ci < MV; ci += nt) {
    const int c = ci / NL, i = ci % NL;
    int im[3];
    node_multi<D, N>(i, im);
    T ad = 0, md = 0;
    for (int nb = 0; nb < NNB; ++nb) {
      const int o[3] = {nb % 3 - 1, (nb / 3) % 3 - 1, nb / 9 - 1};
      bool ok = true;
      int64_t nc = 0, s = 1;
      int ii = 0, si = 1;
      for (int l = 0; l < D; ++l) {
        const int x = cc[l] + o[l], a = im[l] - o[l] * (N - 1);
        if (x < 0 || x >= L.n || a < 0 || a >= N) { ok = false; break; }
        nc += (int64_t)x * s; s *= L.n;
        ii += a * si; si *= N;
      }
      if (!ok) continue;
      const int64_t ec = nc - V.ebase;
      ad += V.EA[ec * (int64_t)MV * MV + (int64_t)(c * NL + ii) * MV + c * NL + ii];
      md += V.EM[ec * (int64_t)NL * NL + (int64_t)ii * NL + ii];
    }
    T Tm[MAXKP1][MAXKP1], Ti[MAXKP1][MAXKP1];
#pragma unroll
    for (int a = 0; a < MAXKP1; ++a)
#pragma unroll
      for (int b = 0; b < MAXKP1; ++b)
        Tm[a][b] = (a < kp1 && b < kp1) ? tb.K[a][b] * md + (a == b ? tb.w[a] * ad : (T)0) : (T)(a == b ? 1 : 0);
    if (!small_inverse<T>(Tm, kp1, Ti)) { *V.status = 1; Ti[0][0] = 0; }
    for (int a = 0; a < kp1; ++a)
      for (int b = 0; b < kp1; ++b) {
        s_ti[(ci * kp1 + a) * kp1 + b] = Ti[a][b];
        blob[(ci * kp1 + a) * kp1 + b] = Ti[a][b];
      }
  }
  // the pressure coupling of the cell
  const T* EB = V.EB + (cell - V.ebase) * (int64_t)npc * MV;
  T* bB = blob + (int64_t)MV * kp1 * kp1;
  for (int e = tid; e < npc * MV; e += nt) bB[e] = EB[e];
  __syncthreads();
  // S[(a,m),(b,m')] = w_a w_b sum_ci B[m][ci] Ti_ci[a][b] B[m'][ci]
  for (int e = tid; e < ns * ns; e += nt) {
    const int row = e / ns, col = e % ns;
    const int a = row / npc, m = row % npc, b = col / npc, mp = col % npc;
    T acc = 0;
    for (int ci = 0; ci < MV; ++ci) acc += EB[m * MV + ci] * s_ti[(ci * kp1 + a) * kp1 + b] * EB[mp * MV + ci];
    s_S[e] = tb.w[a] * tb.w[b] * acc;
  }
  __syncthreads();
  if (!gauss_jordan<T>(s_S, ns, ns, s_piv, s_col)) { if (tid == 0) *V.status = 1; return; }
  T* bS = bB + (int64_t)npc * MV;
  for (int e = tid; e < ns * ns; e += nt) bS[e] = s_S[e];
}

// Dynamic shared memory of one cell slot of k_vanka_apply_diag (blob, right-hand sides, work
// vectors, index list), rounded to 16 bytes.
__host__ __device__ inline size_t diag_slot_bytes(int mv, int npc, int kp1, size_t t) {
  const size_t ms = (size_t)mv + npc;
  const size_t ents = (size_t)diag_blob_entries(mv, npc, kp1) + 3 * (size_t)kp1 * ms;
  return ((ents * t + ms * 8) + 15) & ~(size_t)15;
}

// d[patch] += W~ (modified patch)^{-1} res[patch] for the cells of one colour (W~ = omega on
// velocity, omega_p on pressure DoFs).  One warp per cell, CPB cells per block.
template <typename T, int D, int N>
__global__ void k_vanka_apply_diag(LevelArgs<T> L, const T* __restrict__ blobs, const T* __restrict__ res,
                                   T* __restrict__ d, T omega, T omega_p, Tab<T> tb, ColorInfo ci, int cpb,
                                   SlotStrides zs) {
  blobs += blockIdx.y * zs.inv;
  res += blockIdx.y * zs.vec;
  d += blockIdx.y * zs.vec;
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int npc = tb.npc, kp1 = tb.k + 1, ns = kp1 * npc, ms = MV + npc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nblob = diag_blob_entries(MV, npc, kp1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_raw + (size_t)warp * diag_slot_bytes(MV, npc, kp1, sizeof(T));
  T* sb = reinterpret_cast<T*>(base);                 // blob
  T* rv = sb + nblob;                                 // [kp1][ms] residual on the patch
  T* yv = rv + kp1 * ms;                              // [kp1][ms] y (velocity) / g, p (pressure)
  T* qv = yv + kp1 * ms;                              // [kp1][ms] work
  int64_t* gb = reinterpret_cast<int64_t*>(qv + kp1 * ms);   // [ms] global index at time node 0
  const int cidx = blockIdx.x * cpb + warp;
  if (warp >= cpb || cidx >= ci.count) return;        // whole warps leave; no block barrier below
  int cc[3] = {0, 0, 0};
  decode_color_cell<D>(ci, cidx, cc);
  int64_t cell = 0, s = 1;
  for (int l = 0; l < D; ++l) { cell += (int64_t)cc[l] * s; s *= L.n; }
  const T* src = blobs + cell * nblob;
  for (int64_t e = lane; e < nblob; e += 32) sb[e] = src[e];
  for (int l = lane; l < ms; l += 32) {
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
    for (int a = 0; a < kp1; ++a) rv[a * ms + l] = res[g + a * sa];
  }
  __syncwarp();
  const T* Ti = sb;
  const T* B = sb + (int64_t)MV * kp1 * kp1;
  const T* Si = B + (int64_t)npc * MV;
  // y = A_d^{-1} r_v
  for (int c = lane; c < MV; c += 32)
    for (int a = 0; a < kp1; ++a) {
      T acc = 0;
      for (int b = 0; b < kp1; ++b) acc += Ti[(c * kp1 + a) * kp1 + b] * rv[b * ms + c];
      yv[a * ms + c] = acc;
    }
  __syncwarp();
  // g = (W (x) B) y - r_p, kept in qv's pressure rows
  for (int e = lane; e < ns; e += 32) {
    const int a = e / npc, m = e % npc;
    T acc = 0;
    for (int c = 0; c < MV; ++c) acc += B[m * MV + c] * yv[a * ms + c];
    qv[a * ms + MV + m] = tb.w[a] * acc - rv[a * ms + MV + m];
  }
  __syncwarp();
  // p = S^{-1} g, into yv's pressure rows
  for (int e = lane; e < ns; e += 32) {
    T acc = 0;
    for (int f = 0; f < ns; ++f) acc += Si[e * ns + f] * qv[(f / npc) * ms + MV + f % npc];
    yv[(e / npc) * ms + MV + e % npc] = acc;
  }
  __syncwarp();
  // q = (W (x) B)^T p on the velocity rows, v = y - A_d^{-1} q, and the damped update
  for (int c = lane; c < MV; c += 32) {
    T q[MAXKP1];
    for (int a = 0; a < kp1; ++a) {
      T acc = 0;
      for (int m = 0; m < npc; ++m) acc += B[m * MV + c] * yv[a * ms + MV + m];
      q[a] = tb.w[a] * acc;
    }
    const int64_t g = gb[c];
    for (int a = 0; a < kp1; ++a) {
      T acc = 0;
      for (int b = 0; b < kp1; ++b) acc += Ti[(c * kp1 + a) * kp1 + b] * q[b];
      d[g + a * L.Nv] += omega * (yv[a * ms + c] - acc);
    }
  }
  for (int e = lane; e < ns; e += 32) {
    const int a = e / npc, m = e % npc;
    d[gb[MV + m] + a * L.Np] += omega_p * yv[a * ms + MV + m];
  }
}

}  // namespace stmg
