// Vector kernels (see vec.cuh).  Grid-stride loops sized as a multiple of the SM count;
// reductions in a fixed order (block partial sums, then one block per result).
#include "vec.cuh"
#include "counters.hpp"

namespace stmg {

static inline int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename T>
__global__ void k_axpby(int64_t n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

template <typename T>
cudaError_t vaxpby(int64_t n, T a, const T* x, T b, T* y, cudaStream_t s) {
  k_axpby<T><<<grid_for(n), 256, 0, s>>>(n, a, x, b, y);
  note_launch();
  return cudaGetLastError();
}

template <typename S, typename T>
__global__ void k_copy(int64_t n, const S* __restrict__ x, T* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (T)x[i];
}

template <typename S, typename T>
cudaError_t vcopy(int64_t n, const S* x, T* y, cudaStream_t s) {
  k_copy<S, T><<<grid_for(n), 256, 0, s>>>(n, x, y);
  note_launch();
  return cudaGetLastError();
}

template <typename S, typename T>
__global__ void k_copy_slots(int64_t n, const S* __restrict__ x, int64_t xs, T* __restrict__ y, int64_t ys) {
  x += blockIdx.y * xs;
  y += blockIdx.y * ys;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (T)x[i];
}

template <typename S, typename T>
cudaError_t vcopy_slots(int64_t n, int slots, const S* x, int64_t xs, T* y, int64_t ys, cudaStream_t s) {
  k_copy_slots<S, T><<<dim3(grid_for(n), slots), 256, 0, s>>>(n, x, xs, y, ys);
  note_launch();
  return cudaGetLastError();
}

// Partial dot products of up to DOTS_PER_ROW basis vectors with w per block: w[i] is read once
// for all of them.  Each thread accumulates its strided elements in index order, then the block
// reduces in a fixed tree: the result does not depend on how many vectors share a block.
constexpr int DOTS_PER_ROW = 4;

template <typename T>
__global__ void k_dots_partial(int64_t n, int m, const T* __restrict__ X, int64_t ldx, const T* __restrict__ w,
                               double* __restrict__ part) {
  __shared__ double red[DOTS_PER_ROW][RED_THREADS];
  const int l0 = blockIdx.y * DOTS_PER_ROW;
  const int cnt = m - l0 < DOTS_PER_ROW ? m - l0 : DOTS_PER_ROW;
  double acc[DOTS_PER_ROW] = {0.0, 0.0, 0.0, 0.0};
  const int64_t stride = (int64_t)RED_BLOCKS * RED_THREADS;
  for (int64_t i = blockIdx.x * (int64_t)RED_THREADS + threadIdx.x; i < n; i += stride) {
    const double wi = (double)w[i];
    double xv[DOTS_PER_ROW];
#pragma unroll
    for (int q = 0; q < DOTS_PER_ROW; ++q) xv[q] = q < cnt ? (double)X[(l0 + q) * ldx + i] : 0.0;
#pragma unroll
    for (int q = 0; q < DOTS_PER_ROW; ++q) acc[q] += xv[q] * wi;
  }
#pragma unroll
  for (int q = 0; q < DOTS_PER_ROW; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int q = 0; q < DOTS_PER_ROW; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < cnt) part[(l0 + threadIdx.x) * RED_BLOCKS + blockIdx.x] = red[threadIdx.x][0];
}

__global__ void k_dots_final(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double red[RED_THREADS];
  const int l = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < RED_BLOCKS; i += RED_THREADS) acc += part[l * RED_BLOCKS + i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[l] = red[0];
}

template <typename T>
cudaError_t vdots(int64_t n, int m, const T* X, int64_t ldx, const T* w, double* out, double* scratch,
                  cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  k_dots_partial<T><<<dim3(RED_BLOCKS, (m + DOTS_PER_ROW - 1) / DOTS_PER_ROW), RED_THREADS, 0, s>>>(n, m, X, ldx, w,
                                                                                              scratch);
  note_launch();
  k_dots_final<<<m, RED_THREADS, 0, s>>>(scratch, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_sub_comb(int64_t n, int m, const T* __restrict__ X, int64_t ldx, const double* __restrict__ h,
                           T* __restrict__ w) {
  __shared__ double hs[64];
  if (threadIdx.x < m) hs[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = (double)w[i];
#pragma unroll 8
    for (int l = 0; l < m; ++l) acc -= hs[l] * (double)X[l * ldx + i];
    w[i] = (T)acc;
  }
}

template <typename T>
cudaError_t vsub_comb(int64_t n, int m, const T* X, int64_t ldx, const double* h, T* w, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  if (m > 64) return cudaErrorInvalidValue;
  k_sub_comb<T><<<grid_for(n), 256, 0, s>>>(n, m, X, ldx, h, w);
  note_launch();
  return cudaGetLastError();
}

struct Coef64 { double v[64]; };

__global__ void k_add_comb(int64_t n, int m, const double* __restrict__ Z, int64_t ldz, Coef64 y,
                           double* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[i];
    for (int l = 0; l < m; ++l) acc += y.v[l] * Z[l * ldz + i];
    x[i] = acc;
  }
}

cudaError_t vadd_comb_host(int64_t n, int m, const double* Z, int64_t ldz, const double* y, double* x,
                           cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  if (m > 64) return cudaErrorInvalidValue;
  Coef64 c{};
  for (int l = 0; l < m; ++l) c.v[l] = y[l];
  k_add_comb<<<grid_for(n), 256, 0, s>>>(n, m, Z, ldz, c, x);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void k_scale_inv_dev(int64_t n, const T* __restrict__ x, const double* __restrict__ nrm, T* __restrict__ y) {
  const double f = 1.0 / *nrm;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (T)((double)x[i] * f);
}

template <typename T>
cudaError_t vscale_inv_dev(int64_t n, const T* x, const double* nrm, T* y, cudaStream_t s) {
  k_scale_inv_dev<T><<<grid_for(n), 256, 0, s>>>(n, x, nrm, y);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void k_scale(int64_t n, T a, const T* __restrict__ x, T* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

template <typename T>
cudaError_t vscale(int64_t n, T a, const T* x, T* y, cudaStream_t s) {
  k_scale<T><<<grid_for(n), 256, 0, s>>>(n, a, x, y);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void k_fill(int64_t n, T v, T* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

template <typename T>
cudaError_t vfill(int64_t n, T v, T* x, cudaStream_t s) {
  k_fill<T><<<grid_for(n), 256, 0, s>>>(n, v, x);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_finite(int64_t n, const double* __restrict__ x, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) *flag = 1;
}

cudaError_t vfinite(int64_t n, const double* x, int* flag, cudaStream_t s) {
  k_finite<<<grid_for(n), 256, 0, s>>>(n, x, flag);
  note_launch();
  return cudaGetLastError();
}

template cudaError_t vaxpby<float>(int64_t, float, const float*, float, float*, cudaStream_t);
template cudaError_t vaxpby<double>(int64_t, double, const double*, double, double*, cudaStream_t);
template cudaError_t vcopy<double, float>(int64_t, const double*, float*, cudaStream_t);
template cudaError_t vcopy<float, double>(int64_t, const float*, double*, cudaStream_t);
template cudaError_t vcopy<double, double>(int64_t, const double*, double*, cudaStream_t);
template cudaError_t vcopy<float, float>(int64_t, const float*, float*, cudaStream_t);
template cudaError_t vcopy_slots<double, float>(int64_t, int, const double*, int64_t, float*, int64_t, cudaStream_t);
template cudaError_t vcopy_slots<float, double>(int64_t, int, const float*, int64_t, double*, int64_t, cudaStream_t);
template cudaError_t vcopy_slots<double, double>(int64_t, int, const double*, int64_t, double*, int64_t, cudaStream_t);
template cudaError_t vdots<float>(int64_t, int, const float*, int64_t, const float*, double*, double*, cudaStream_t);
template cudaError_t vdots<double>(int64_t, int, const double*, int64_t, const double*, double*, double*, cudaStream_t);
template cudaError_t vsub_comb<float>(int64_t, int, const float*, int64_t, const double*, float*, cudaStream_t);
template cudaError_t vsub_comb<double>(int64_t, int, const double*, int64_t, const double*, double*, cudaStream_t);
template cudaError_t vscale_inv_dev<double>(int64_t, const double*, const double*, double*, cudaStream_t);
template cudaError_t vscale_inv_dev<float>(int64_t, const float*, const double*, float*, cudaStream_t);
template cudaError_t vscale<float>(int64_t, float, const float*, float*, cudaStream_t);
template cudaError_t vscale<double>(int64_t, double, const double*, double*, cudaStream_t);
template cudaError_t vfill<float>(int64_t, float, float*, cudaStream_t);
template cudaError_t vfill<double>(int64_t, double, double*, cudaStream_t);

}  // namespace stmg
