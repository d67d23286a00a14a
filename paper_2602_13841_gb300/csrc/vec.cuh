// Vector kernels on device buffers: copies, casts, axpy, deterministic dot products (fixed
// two-stage reduction order, no atomics) and the CGS2 building blocks of FGMRES.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace stmg {

constexpr int RED_BLOCKS = 1216;     // 8 x 152 SMs: partial sums per dot product
constexpr int RED_THREADS = 256;

// y = a*x + b*y
template <typename T>
cudaError_t vaxpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t s);
// y = x (element type conversion allowed)
template <typename S, typename T>
cudaError_t vcopy(int64_t n, const S* x, T* y, cudaStream_t s);
// y_j = x_j (n entries) for j < slots, x_j = x + j xs, y_j = y + j ys (one launch)
template <typename S, typename T>
cudaError_t vcopy_slots(int64_t n, int slots, const S* x, int64_t xs, T* y, int64_t ys, cudaStream_t s);
// out[l] = sum_i X[l*ldx + i] * w[i], l < m  (device scalars, double); scratch >= m*RED_BLOCKS doubles
template <typename T>
cudaError_t vdots(int64_t n, int m, const T* X, int64_t ldx, const T* w, double* out, double* scratch,
                  cudaStream_t s);
// w -= sum_l h[l] * X[l*ldx + :], h on the device (double), l < m
template <typename T>
cudaError_t vsub_comb(int64_t n, int m, const T* X, int64_t ldx, const double* h, T* w, cudaStream_t s);
// x += sum_l y[l] * Z[l*ldz + :] with host coefficients copied by value (m <= 64)
cudaError_t vadd_comb_host(int64_t n, int m, const double* Z, int64_t ldz, const double* y, double* x,
                           cudaStream_t s);
// y = x * (1 / *nrm) where nrm is a device scalar
template <typename T>
cudaError_t vscale_inv_dev(int64_t n, const T* x, const double* nrm, T* y, cudaStream_t s);
// y = a * x
template <typename T>
cudaError_t vscale(int64_t n, T a, const T* x, T* y, cudaStream_t s);
// set x[i] = v for i in [0, n)
template <typename T>
cudaError_t vfill(int64_t n, T v, T* x, cudaStream_t s);
// NaN / Inf check: *flag = 1 if any entry of x is not finite
cudaError_t vfinite(int64_t n, const double* x, int* flag, cudaStream_t s);

}  // namespace stmg
