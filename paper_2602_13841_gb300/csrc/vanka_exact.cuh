// Exact space-time Vanka patches: S_K = R_K J R_K^T with the convection Jacobian of every time
// node a evaluated at that node's own velocity V^a (Eq. JacobianLocal2), the matrix that the
// midpoint surrogate of Sec. 4.3 (Eq. DefTildeHn, DefVnAst) approximates.  The spatial cores of
// the time nodes differ, so the patch does not split by a time diagonalisation: it is assembled
// whole, (k+1) m_s square,
//     S_K = [ K^tau (x) M + blockdiag_a(w_a A_a) ,  blockdiag_a(w_a B^T) ]
//           [ blockdiag_a(w_a B)                 ,  0                    ]
// (patch ordering: time node a, then the spatial patch DoF), inverted by Gauss-Jordan elimination
// with partial pivoting in shared memory, and stored column-major with the padded stride of
// inv_stride.  Supported where the whole patch fits shared memory (2D; 3D Q2/P1 up to DG(1)).
// The comparison with the surrogate is the Lemma's question: how much the single-time-point
// patch costs in iterations, against (k+1) element-matrix passes and a (k+1)^3 times larger
// factorisation per rebuild.
#pragma once
#include "vanka.cuh"

namespace stmg {

// Shared memory of k_patch_exact: S (mst^2), the assembled velocity block of one time node (MV^2),
// the assembled scalar mass (NL^2), a pivot column and the pivot rows.
__host__ __device__ inline size_t patch_exact_smem(int mst, int mv, int nl, size_t es) {
  return es * ((size_t)mst * mst + (size_t)mv * mv + (size_t)nl * nl + mst) + sizeof(int) * mst + 16;
}

// One block per cell.  EA holds the velocity element blocks of time node a at EA + a * V.ea_tstride.
template <typename T, int D, int N>
__global__ void k_patch_exact(VankaArgs<T> V, Tab<T> tb, int64_t ea_tstride, int64_t c0, int64_t c1) {
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int npc = tb.npc, kp1 = tb.k + 1, ms = MV + npc, mst = kp1 * ms;
  const int st = inv_stride(mst, (int)sizeof(T));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);            // [mst][mst] row-major
  T* Ap = S + mst * mst;                            // [MV][MV]
  T* Mp = Ap + MV * MV;                             // [NL][NL]
  T* col = Mp + NL * NL;                            // [mst]
  int* piv = reinterpret_cast<int*>(col + mst);     // [mst]
  const int64_t cell = c0 + blockIdx.x;
  if (cell >= c1) return;
  const LevelArgs<T>& L = V.L;
  int cc[3] = {0, 0, 0};
  cell_coords<D>(cell, L.n, cc);
  const int tid = threadIdx.x, nt = blockDim.x;
  // neighbour sums over the cells sharing both nodes of an entry (for_shared_cells)
  for (int ent = tid; ent < NL * NL; ent += nt) {
    const int i = ent / NL, j = ent % NL;
    int im[3], jm[3];
    node_multi<D, N>(i, im);
    node_multi<D, N>(j, jm);
    T acc = 0;
    for_shared_cells<D, N>(cc, L.n, im, jm, [&](int64_t nc, int ii, int jj) {
      acc += V.EM[(nc - V.ebase) * (int64_t)NL * NL + (int64_t)ii * NL + jj];
    });
    Mp[ent] = acc;
  }
  __syncthreads();
  // temporal mass coupling and the pressure coupling of every time node
  const T* EB = V.EB + (cell - V.ebase) * (int64_t)npc * MV;
  for (int ent = tid; ent < mst * mst; ent += nt) {
    const int row = ent / mst, cl = ent % mst;
    const int a = row / ms, lr = row % ms, b = cl / ms, lc = cl % ms;
    T v = 0;
    if (lr < MV && lc < MV) {
      if (lr / NL == lc / NL) v = tb.K[a][b] * Mp[(lr % NL) * NL + (lc % NL)];
    } else if (a == b && lr < MV) {
      v = tb.w[a] * EB[(lc - MV) * MV + lr];
    } else if (a == b && lc < MV) {
      v = tb.w[a] * EB[(lr - MV) * MV + lc];
    }
    S[ent] = v;
  }
  __syncthreads();
  // the velocity block of each time node at its own state
  for (int a = 0; a < kp1; ++a) {
    const T* EA = V.EA + (int64_t)a * ea_tstride;
    for (int ent = tid; ent < MV * MV; ent += nt) {
      const int row = ent / MV, cl = ent % MV;
      const int c = row / NL, i = row % NL, e = cl / NL, j = cl % NL;
      int im[3], jm[3];
      node_multi<D, N>(i, im);
      node_multi<D, N>(j, jm);
      T acc = 0;
      for_shared_cells<D, N>(cc, L.n, im, jm, [&](int64_t nc, int ii, int jj) {
        acc += EA[(nc - V.ebase) * (int64_t)MV * MV + (int64_t)(c * NL + ii) * MV + e * NL + jj];
      });
      S[(a * ms + row) * mst + a * ms + cl] += tb.w[a] * acc;
    }
    __syncthreads();
  }
  if (!gauss_jordan<T>(S, mst, mst, piv, col)) { if (tid == 0) *V.status = 1; return; }
  T* inv = V.inv + cell * (int64_t)mst * st;
  for (int ent = tid; ent < mst * st; ent += nt) {
    const int j = ent / st, i = ent % st;           // column-major: inv[j][i] = S^{-1}[i][j]
    inv[ent] = i < mst ? S[i * mst + j] : (T)0;
  }
}

// Dynamic shared memory of k_vanka_apply_exact: [inverse | residual (mst) | global index (ms) | mbarrier].
__host__ __device__ inline size_t apply_exact_smem(int mst, int ms, size_t t) {
  const size_t blob = ((size_t)mst * inv_stride(mst, (int)t) * t + 127) & ~(size_t)127;
  return blob + (((size_t)mst * t + 7) & ~(size_t)7) + (size_t)ms * 8 + 16;
}

// d[patch] += W~ S_K^{-1} res[patch] for the cells of one colour; one block per cell, thread i owns
// patch row i (time node i / m_s, spatial DoF i % m_s).  The inverse is staged by bulk copies on an
// mbarrier with the bounded wait of k_vanka_apply.
template <typename T, int D, int N>
__global__ void k_vanka_apply_exact(LevelArgs<T> L, const T* __restrict__ inv, const T* __restrict__ res,
                                    T* __restrict__ d, T omega, T omega_p, int kp1, int npc, ColorInfo ci,
                                    int* __restrict__ wstat, unsigned extra_tx, SlotStrides zs) {
  inv += blockIdx.y * zs.inv;
  res += blockIdx.y * zs.vec;
  d += blockIdx.y * zs.vec;
  constexpr int NL = Shape<D, N>::Q;
  constexpr int MV = D * NL;
  const int ms = MV + npc, mst = kp1 * ms, st = inv_stride(mst, (int)sizeof(T));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t blob = ((size_t)mst * st * sizeof(T) + 127) & ~(size_t)127;
  T* sinv = reinterpret_cast<T*>(smem_raw);
  T* rt = reinterpret_cast<T*>(smem_raw + blob);
  int64_t* gb = reinterpret_cast<int64_t*>(smem_raw + blob + (((size_t)mst * sizeof(T) + 7) & ~(size_t)7));
  uint64_t* bar = reinterpret_cast<uint64_t*>(gb + ms);
  const int cidx = blockIdx.x;
  if (cidx >= ci.count) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  int cc[3] = {0, 0, 0};
  decode_color_cell<D>(ci, cidx, cc);
  int64_t cell = 0, s = 1;
  for (int l = 0; l < D; ++l) { cell += (int64_t)cc[l] * s; s *= L.n; }
  const uint32_t b = smem_addr(bar);
  const uint32_t bytes = (uint32_t)((size_t)mst * st * sizeof(T));
  if (tid == 0) {
    mbar_init(b, 1);
    mbar_expect_tx(b, bytes + extra_tx);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(inv + cell * (int64_t)mst * st);
    for (uint32_t o = 0; o < bytes; o += kBulkChunk) {
      const uint32_t n = bytes - o < (uint32_t)kBulkChunk ? bytes - o : (uint32_t)kBulkChunk;
      bulk_g2s(smem_addr(smem_raw + o), src + o, n, b);
    }
  }
  for (int l = tid; l < ms; l += nt) {
    int64_t g;
    if (l < MV) {
      const int c = l / NL, i = l % NL;
      g = c * L.nnodes + global_node<D>(L.N1, cc, N - 1, i, N);
    } else {
      g = (int64_t)kp1 * L.Nv + cell * npc + (l - MV);
    }
    gb[l] = g;
  }
  __syncthreads();
  for (int i = tid; i < mst; i += nt) {
    const int a = i / ms, l = i % ms;
    rt[i] = res[gb[l] + (int64_t)a * (l < MV ? L.Nv : L.Np)];
  }
  __syncthreads();
  if (!mbar_wait_bounded(b, 0, kWaitLimit)) {
    if (tid == 0) atomicExch(wstat, 1);
    mbar_wait_bounded(b, 0, kWaitLimit);
    return;
  }
  for (int i = tid; i < mst; i += nt) {
    T acc = 0;
    for (int j = 0; j < mst; ++j) acc += sinv[j * st + i] * rt[j];
    const int a = i / ms, l = i % ms;
    const int64_t g = gb[l] + (int64_t)a * (l < MV ? L.Nv : L.Np);
    d[g] += (l < MV ? omega : omega_p) * acc;
  }
}

}  // namespace stmg
