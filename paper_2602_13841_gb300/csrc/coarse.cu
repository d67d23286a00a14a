// Coarsest-level direct solve (Sec. 4.2, "solved directly").  The coarse Jacobian is assembled
// column by column by a batched matrix-free apply to the identity, bordered with one mean-zero
// pressure row and column per time node (pure Dirichlet: pressure in L^2_0), inverted once per
// smoother build by single-block Gauss-Jordan in FP32, and applied with two steps of FP64
// iterative refinement against the FP64 bordered matrix, so the coarse solution is FP64-accurate.
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

__global__ void k_to_rowmajor32(const double* __restrict__ A, float* __restrict__ S, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int row = (int)(e / n), col = (int)(e % n);
    S[e] = (float)A[(int64_t)col * n + row];
  }
}

__global__ void k_gj_single(float* S, int n, float* col, int* piv, int* status) {
  bool ok = gauss_jordan<float>(S, n, n, piv, col);
  if (!ok && threadIdx.x == 0) *status = 1;
}

__global__ void k_transpose32(float* S, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), j = (int)(e % n);
    if (i < j) { float t = S[(int64_t)i * n + j]; S[(int64_t)i * n + j] = S[(int64_t)j * n + i]; S[(int64_t)j * n + i] = t; }
  }
}

cudaError_t coarse_invert(const double* A, float* Ainv, float* col, int* piv, int Nb, int* status,
                          cudaStream_t s) {
  k_to_rowmajor32<<<152 * 4, 256, 0, s>>>(A, Ainv, Nb);
  note_launch();
  k_gj_single<<<1, 1024, 0, s>>>(Ainv, Nb, col, piv, status);
  k_transpose32<<<152 * 4, 256, 0, s>>>(Ainv, Nb);    // row-major inverse -> column-major
  return cudaGetLastError();
}

template <typename TA>
__global__ void k_gemv_cm(const TA* __restrict__ A, int n, const double* __restrict__ x, double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc += (double)A[(int64_t)j * n + i] * x[j];
    y[i] = acc;
  }
}

cudaError_t gemv_cm(const double* A, int n, const double* x, double* y, cudaStream_t s) {
  k_gemv_cm<double><<<(n + 127) / 128, 128, 0, s>>>(A, n, x, y);
  note_launch();
  return cudaGetLastError();
}

cudaError_t gemv_cm(const float* A, int n, const double* x, double* y, cudaStream_t s) {
  k_gemv_cm<float><<<(n + 127) / 128, 128, 0, s>>>(A, n, x, y);
  note_launch();
  return cudaGetLastError();
}

}  // namespace stmg
