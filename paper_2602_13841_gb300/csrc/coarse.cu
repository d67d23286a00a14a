// Coarsest-level direct solve (Sec. 4.2, "solved directly").  The coarse Jacobian is assembled
// column by column by a batched matrix-free apply to the identity, bordered with one mean-zero
// pressure row and column per time node (pure Dirichlet: pressure in L^2_0), inverted once per
// smoother build by Gauss-Jordan elimination with partial pivoting in FP64, and applied in FP64
// with one step of iterative refinement against the bordered matrix.
#include "mg.hpp"
#include "op_launch.cuh"
#include "vanka.cuh"
#include "counters.hpp"

namespace stmg {

// A (Nb x Nb, column-major) = [[J, C^T], [C, 0]] with C_a = (pressure part of M e_a), e_a the
// constant pressure at time node a.  J: N x N column-major.
__global__ void k_border_copy(const double* __restrict__ J, double* __restrict__ A, int N, int Nb) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)Nb * Nb;
       e += (int64_t)gridDim.x * blockDim.x) {
    int col = (int)(e / Nb), row = (int)(e % Nb);
    A[e] = (col < N && row < N) ? J[(int64_t)col * N + row] : 0.0;
  }
}

__global__ void k_const_pressure(double* __restrict__ e, int64_t poff, int64_t Np, int npc, int a, int N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t rel = i - poff - (int64_t)a * Np;
    e[i] = (rel >= 0 && rel < Np && rel % npc == 0) ? 1.0 : 0.0;
  }
}

__global__ void k_border_rows(const double* __restrict__ Me, double* __restrict__ A, int N, int Nb, int a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    A[(int64_t)(N + a) * Nb + i] = Me[i];     // column N+a, row i   (C^T)
    A[(int64_t)i * Nb + N + a] = Me[i];       // column i, row N+a   (C)
  }
}

cudaError_t coarse_border(const Level& lv, const Problem& pb, const double* J, double* A, int N, int Nb,
                          cudaStream_t s) {
  k_border_copy<<<152 * 4, 256, 0, s>>>(J, A, N, Nb);
  note_launch();
  // scratch: the two columns after J (caller allocates Nb*Nb + 2*N for J's buffer)
  double* e = const_cast<double*>(J) + (int64_t)N * N;
  double* Me = e + N;
  for (int a = 0; a <= lv.k; ++a) {
    k_const_pressure<<<64, 256, 0, s>>>(e, (int64_t)(lv.k + 1) * lv.Nv, lv.Np, lv.npc, a, N);
  note_launch();
    cudaError_t err = launch_operator<double>(lv, pb, OP_MASS, 0.0, e, nullptr, nullptr, Me, s);
    if (err != cudaSuccess) return err;
    k_border_rows<<<64, 256, 0, s>>>(Me, A, N, Nb, a);
  note_launch();
  }
  return cudaGetLastError();
}

__global__ void k_to_rowmajor(const double* __restrict__ A, double* __restrict__ S, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int row = (int)(e / n), col = (int)(e % n);
    S[e] = A[(int64_t)col * n + row];
  }
}

__global__ void k_gj_single(double* S, int n, double* col, int* piv, int* status) {
  bool ok = gauss_jordan<double>(S, n, n, piv, col);
  if (!ok && threadIdx.x == 0) *status = 1;
}

__global__ void k_transpose(double* S, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    if (i < j) { double t = S[(int64_t)i * n + j]; S[(int64_t)i * n + j] = S[(int64_t)j * n + i]; S[(int64_t)j * n + i] = t; }
  }
}

// Gauss-Jordan step p of a large coarse matrix (row-major, in place), the same arithmetic as
// gauss_jordan spread over launches: k_gj_pivot (one block) picks and swaps the pivot row,
// scales it and moves column p into `col`; k_gj_elim (all SMs) updates the other rows; after the
// last step k_gj_unswap (one block) undoes the column exchanges.  A zero pivot sets *status and
// turns the remaining steps into no-ops.
__global__ void k_gj_pivot(double* S, int n, int p, double* col, int* piv, int* status) {
  __shared__ int s_r;
  __shared__ double s_best[32];
  __shared__ int s_idx[32];
  if (*status) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  double best = -1.0; int bi = p;
  for (int i = p + tid; i < n; i += nt) {
    const double a = fabs(S[(int64_t)i * n + p]);
    if (a > best || (a == best && i < bi)) { best = a; bi = i; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if ((tid & 31) == 0) { s_best[tid >> 5] = best; s_idx[tid >> 5] = bi; }
  __syncthreads();
  if (tid < 32) {
    best = tid < (nt >> 5) ? s_best[tid] : -1.0;
    bi = tid < (nt >> 5) ? s_idx[tid] : p;
    for (int off = 16; off > 0; off >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (tid == 0) { s_r = bi; piv[p] = bi; if (!(best > 0.0)) *status = 1; }
  }
  __syncthreads();
  if (*status) return;
  const int r = s_r;
  if (r != p)
    for (int j = tid; j < n; j += nt) {
      const double t = S[(int64_t)p * n + j]; S[(int64_t)p * n + j] = S[(int64_t)r * n + j]; S[(int64_t)r * n + j] = t;
    }
  __syncthreads();
  const double pinv = 1.0 / S[(int64_t)p * n + p];
  __syncthreads();
  for (int j = tid; j < n; j += nt) S[(int64_t)p * n + j] = (j == p) ? pinv : S[(int64_t)p * n + j] * pinv;
  for (int i = tid; i < n; i += nt) {
    col[i] = (i == p) ? 0.0 : S[(int64_t)i * n + p];
    if (i != p) S[(int64_t)i * n + p] = 0.0;
  }
}

__global__ void k_gj_elim(double* S, int n, int p, const double* __restrict__ col, const int* status) {
  if (*status) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i != p) S[e] -= col[i] * S[(int64_t)p * n + j];
  }
}

__global__ void k_gj_unswap(double* S, int n, const int* __restrict__ piv, const int* status) {
  if (*status) return;
  for (int p = n - 1; p >= 0; --p) {
    const int r = piv[p];
    if (r != p)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double t = S[(int64_t)i * n + p]; S[(int64_t)i * n + p] = S[(int64_t)i * n + r]; S[(int64_t)i * n + r] = t;
      }
    __syncthreads();
  }
}

cudaError_t coarse_invert(const double* A, double* Ainv, double* col, int* piv, int Nb, int* status,
                          cudaStream_t s) {
  k_to_rowmajor<<<152 * 4, 256, 0, s>>>(A, Ainv, Nb);
  note_launch();
  if (Nb <= 512) {
    k_gj_single<<<1, 1024, 0, s>>>(Ainv, Nb, col, piv, status);
    note_launch();
  } else {
    // large coarse systems (3D): one pivot launch and one all-SM elimination launch per step
    for (int p = 0; p < Nb; ++p) {
      k_gj_pivot<<<1, 1024, 0, s>>>(Ainv, Nb, p, col, piv, status);
      k_gj_elim<<<152 * 4, 256, 0, s>>>(Ainv, Nb, p, col, status);
    }
    k_gj_unswap<<<1, 1024, 0, s>>>(Ainv, Nb, piv, status);
    note_launch(2 * Nb + 1);
  }
  k_transpose<<<152 * 4, 256, 0, s>>>(Ainv, Nb);      // row-major inverse -> column-major
  note_launch();
  return cudaGetLastError();
}

template <typename TA>
__global__ void k_gemv_cm(const TA* __restrict__ A, int n, const double* __restrict__ x, double* __restrict__ y) {
  A += (int64_t)blockIdx.y * n * n;           // blockIdx.y: independent slot
  x += (int64_t)blockIdx.y * n;
  y += (int64_t)blockIdx.y * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += (double)A[(int64_t)j * n + i] * x[j];
    y[i] = acc;
  }
}

cudaError_t gemv_cm(const double* A, int n, const double* x, double* y, cudaStream_t s, int slots) {
  k_gemv_cm<double><<<dim3((n + 127) / 128, slots), 128, 0, s>>>(A, n, x, y);
  note_launch();
  return cudaGetLastError();
}


}  // namespace stmg
