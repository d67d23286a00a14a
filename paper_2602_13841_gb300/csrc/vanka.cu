// Vanka smoother launchers (kernels in vanka.cuh).
#include <type_traits>

#include "mg.hpp"
#include "op_launch.cuh"
#include "vanka.cuh"
#include "vec.cuh"
#include "counters.hpp"

namespace stmg {

size_t vanka_patch_size(const Level& lv) {
  int nl = 1;
  for (int l = 0; l < lv.d; ++l) nl *= (lv.r + 2);
  return (size_t)(lv.k + 1) * (lv.d * nl + lv.npc);
}

size_t vanka_elem_size(const Level& lv, int which) {
  size_t nl = 1;
  for (int l = 0; l < lv.d; ++l) nl *= (lv.r + 2);
  size_t mv = lv.d * nl;
  if (which == 0) return mv * mv;
  if (which == 1) return (size_t)lv.npc * mv;
  return nl * nl;
}

template <int D, int N>
static size_t elem_smem(size_t es) {
  constexpr int Q = Shape<D, N>::Q, NL = Q, NF = Shape<D, N>::NF;
  constexpr int FSZ = NF * (2 + 2 * D) + 2 * NF * NL;
  return es * (Q * NL * D + Q * NL + Q + Q * D + D * NL + D * FSZ + 8 + 24);
}

static size_t patch_smem(const Level& lv, size_t es) {
  size_t m = vanka_patch_size(lv);
  size_t nl = 1;
  for (int l = 0; l < lv.d; ++l) nl *= (lv.r + 2);
  size_t mv = lv.d * nl;
  return es * (m * m + mv * mv + nl * nl + m) + sizeof(int) * m;
}

static size_t elem_smem_any(const Level& lv, size_t es) {
  int N = lv.r + 2;
  if (lv.d == 2) return N == 3 ? elem_smem<2, 3>(es) : N == 4 ? elem_smem<2, 4>(es) : elem_smem<2, 5>(es);
  return N == 3 ? elem_smem<3, 3>(es) : N == 4 ? elem_smem<3, 4>(es) : elem_smem<3, 5>(es);
}

bool vanka_supported(const Level& lv, size_t es) {
  const size_t lim = 227 * 1024;
  return patch_smem(lv, es) <= lim && elem_smem_any(lv, es) <= lim;
}

// v* = sum_a phi_a(t*) V^a
template <typename T>
__global__ void k_midpoint(const T* __restrict__ U, T* __restrict__ vs, int64_t Nv, int kp1, Tab<T> tb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nv; i += (int64_t)gridDim.x * blockDim.x) {
    T acc = 0;
    for (int a = 0; a < kp1; ++a) acc += tb.phi_mid[a] * U[a * Nv + i];
    vs[i] = acc;
  }
}

template <typename T, int D, int N>
static cudaError_t build_dn(const Level& lv, const Problem& pb, const T* U, T* vstar, T* EA, T* EB, T* EM,
                            T* inv, void* invh, float* scale, int* status, cudaStream_t s) {
  Tab<T> tb = make_tab<T>(lv.tabs, pb.tau);
  int64_t ncells = lv.Np / lv.npc;
  int64_t g = (lv.Nv + 255) / 256; if (g > 152 * 8) g = 152 * 8;
  k_midpoint<T><<<(int)g, 256, 0, s>>>(U, vstar, lv.Nv, lv.k + 1, tb);
  VankaArgs<T> V{level_args<T>(lv, pb, 0.0), vstar, EA, EB, EM, inv, (__half*)invh, scale, status};
  size_t es = elem_smem<D, N>(sizeof(T));
  cudaError_t e = cudaFuncSetAttribute(k_elem<T, D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)es);
  if (e != cudaSuccess) return e;
  k_elem<T, D, N><<<(unsigned)ncells, 256, es, s>>>(V, tb, ncells);
  size_t ps = patch_smem(lv, sizeof(T));
  e = cudaFuncSetAttribute(k_patch<T, D, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps);
  if (e != cudaSuccess) return e;
  k_patch<T, D, N><<<(unsigned)ncells, 256, ps, s>>>(V, tb, ncells);
  note_launch(3);
  return cudaGetLastError();
}

template <typename T>
cudaError_t vanka_build(const Level& lv, const Problem& pb, const T* U, T* vstar, T* EA, T* EB, T* EM,
                        T* inv, void* invh, float* scale, int* status, cudaStream_t s) {
  if (!vanka_supported(lv, sizeof(T))) return cudaErrorNotSupported;
  const int N = lv.r + 2;
#define STMG_B(DD, NN) return build_dn<T, DD, NN>(lv, pb, U, vstar, EA, EB, EM, inv, invh, scale, status, s)
  if (lv.d == 2) { if (N == 3) STMG_B(2, 3); if (N == 4) STMG_B(2, 4); if (N == 5) STMG_B(2, 5); }
  else { if (N == 3) STMG_B(3, 3); if (N == 4) STMG_B(3, 4); }
#undef STMG_B
  return cudaErrorNotSupported;
}

template <typename T, typename SI, int D, int N>
static void apply_rows(const Level& lv, const Problem& pb, const SI* inv, const float* scale, const T* res, T* d,
                       double omega, double omega_p, const ColorInfo& ci, cudaStream_t s) {
  // threads per cell: the patch rows at RR rows per thread, rounded up to whole warps; cells
  // per block: as many as fit 128 threads (at least one)
  const int m = (int)vanka_patch_size(lv), mr = (m + 1) & ~1;
  const int rows = (m + InvRows<SI>::RR - 1) / InvRows<SI>::RR;
  const int tpc = ((rows + 31) / 32) * 32;
  const int cpb = tpc >= 128 ? 1 : 128 / tpc;
  const size_t smem = (size_t)cpb * (mr * sizeof(T) + m * sizeof(int64_t));
  const unsigned blocks = (unsigned)((ci.count + cpb - 1) / cpb);
  k_vanka_apply<T, SI, D, N><<<blocks, tpc * cpb, smem, s>>>(level_args<T>(lv, pb, 0.0), inv, scale, res, d,
                                                             (T)omega, (T)omega_p, lv.k + 1, lv.npc, tpc, ci);
}

template <typename T, int D, int N>
static cudaError_t apply_dn(const Level& lv, const Problem& pb, const T* inv, const void* invh, const float* scale,
                            const T* res, T* d, double omega, double omega_p, int color, cudaStream_t s) {
  const ColorInfo& ci = lv.colors[color];
  if (ci.count == 0) return cudaSuccess;
  if (invh)
    apply_rows<T, __half, D, N>(lv, pb, (const __half*)invh, scale, res, d, omega, omega_p, ci, s);
  else
    apply_rows<T, T, D, N>(lv, pb, inv, nullptr, res, d, omega, omega_p, ci, s);
  note_launch();
  return cudaGetLastError();
}

size_t vanka_inv_entries(const Level& lv) {
  const size_t m = vanka_patch_size(lv);
  return m * (size_t)inv_stride((int)m);
}

template <typename T>
cudaError_t vanka_apply(const Level& lv, const Problem& pb, const T* inv, const void* invh, const float* scale,
                        const T* res, T* d, double omega, double omega_p, int color, cudaStream_t s) {
  const int N = lv.r + 2;
#define STMG_A(DD, NN) return apply_dn<T, DD, NN>(lv, pb, inv, invh, scale, res, d, omega, omega_p, color, s)
  if (lv.d == 2) { if (N == 3) STMG_A(2, 3); if (N == 4) STMG_A(2, 4); if (N == 5) STMG_A(2, 5); }
  else { if (N == 3) STMG_A(3, 3); if (N == 4) STMG_A(3, 4); }
#undef STMG_A
  return cudaErrorNotSupported;
}

template cudaError_t vanka_build<float>(const Level&, const Problem&, const float*, float*, float*, float*, float*,
                                        float*, void*, float*, int*, cudaStream_t);
template cudaError_t vanka_build<double>(const Level&, const Problem&, const double*, double*, double*, double*,
                                         double*, double*, void*, float*, int*, cudaStream_t);
template cudaError_t vanka_apply<float>(const Level&, const Problem&, const float*, const void*, const float*,
                                        const float*, float*, double, double, int, cudaStream_t);
template cudaError_t vanka_apply<double>(const Level&, const Problem&, const double*, const void*, const float*,
                                         const double*, double*, double, double, int, cudaStream_t);

}  // namespace stmg
