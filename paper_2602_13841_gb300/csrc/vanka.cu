// Vanka smoother: sizes, support checks and the dispatch of the build and sweep launches to the
// per-dimension translation units (kernels in vanka.cuh, vanka_diag.cuh, vanka_exact.cuh; launch
// templates in vanka_launch.cuh).
#include "vanka_launch.cuh"

namespace stmg {

// instantiated in vanka_d{2,3}_{f32,f64}.cu
#define STMG_EXTERN(T, D)                                                                                        \
  extern template cudaError_t vanka_build_dim<T, D>(const Level&, const Problem&, const T*, T*, T*, T*, T*, T*,  \
                                                    void*, float*, int*, T*, cudaStream_t);                       \
  extern template cudaError_t vanka_apply_dim<T, D>(const Level&, const Problem&, const T*, const void*,         \
                                                    const float*, const T*, T*, double, double, int, int*,       \
                                                    cudaStream_t, unsigned, int);
STMG_EXTERN(float, 2)
STMG_EXTERN(double, 2)
STMG_EXTERN(float, 3)
STMG_EXTERN(double, 3)
#undef STMG_EXTERN

size_t vanka_spatial_size(const Level& lv) {
  int nl = 1;
  for (int l = 0; l < lv.d; ++l) nl *= (lv.r + 2);
  return (size_t)(lv.d * nl + lv.npc);
}

size_t vanka_patch_size(const Level& lv) { return (size_t)(lv.k + 1) * vanka_spatial_size(lv); }

size_t vanka_elem_size(const Level& lv, int which) {
  size_t nl = 1;
  for (int l = 0; l < lv.d; ++l) nl *= (lv.r + 2);
  size_t mv = lv.d * nl;
  if (which == 0) return mv * mv;
  if (which == 1) return (size_t)lv.npc * mv;
  return nl * nl;
}

bool vanka_supported(const Level& lv, size_t es) {
  const size_t lim = 227 * 1024;
  const size_t ms = vanka_spatial_size(lv);
  if (lv.smoother == 1) return patch_diag_smem(lv, es) <= lim;
  if (lv.smoother == 2) {
    const int mst = (lv.k + 1) * (int)ms, mv = (int)(ms - lv.npc), nl = mv / lv.d;
    return patch_exact_smem(mst, mv, nl, es) <= lim && apply_exact_smem(mst, (int)ms, es) <= lim;
  }
  return es * 2 * ms + sizeof(int) * ms + 16 <= lim;
}

// Cells whose element matrices the build scratch holds at once (whole level if smaller): at most
// chunk_cells cells and at most 8 GiB of FP64 element matrices (3D Q4/P3: 1.3 MB per cell).
size_t vanka_elem_cells(const Level& lv) {
  const size_t ncells = lv.Np / lv.npc, plane = ncells / lv.n;
  size_t nl = 1;
  for (int l = 0; l < lv.d; ++l) nl *= (lv.r + 2);
  const size_t mv = lv.d * nl, per = 8 * (mv * mv + (size_t)lv.npc * mv + nl * nl);
  size_t cap = (size_t)lv.chunk_cells;
  if (cap * per > ((size_t)8 << 30)) cap = ((size_t)8 << 30) / per;
  if (ncells <= cap) return ncells;
  const size_t planes = cap / plane > 3 ? cap / plane : 3;     // a chunk plus its two halo planes
  return planes * plane < ncells ? planes * plane : ncells;
}

size_t vanka_work_entries(const Level& lv, size_t es) {
  const size_t pw = (lv.smoother == 1 || patch_onchip(lv, es)) ? 0 : (size_t)kWorkSlots * work_slot(lv);
  const size_t ew = elem_onchip(lv, es) ? 0 : (size_t)kWorkSlots * elem_table_any(lv);
  return pw > ew ? pw : ew;
}

size_t vanka_inv_entries(const Level& lv, int es) {
  const size_t ms = vanka_spatial_size(lv);
  if (lv.smoother == 1) return (size_t)diag_blob_entries((int)(ms - lv.npc), lv.npc, lv.k + 1);
  if (lv.smoother == 2) {
    const int mst = (lv.k + 1) * (int)ms;
    return (size_t)mst * (size_t)inv_stride(mst, es);
  }
  return (size_t)(lv.k + 1) * ms * (size_t)inv_stride((int)ms, es);
}

template <typename T>
cudaError_t vanka_build(const Level& lv, const Problem& pb, const T* U, T* vstar, T* EA, T* EB, T* EM,
                        T* inv, void* invh, float* scale, int* status, T* work, cudaStream_t s) {
  if (!vanka_supported(lv, sizeof(T))) return cudaErrorNotSupported;
  return lv.d == 2 ? vanka_build_dim<T, 2>(lv, pb, U, vstar, EA, EB, EM, inv, invh, scale, status, work, s)
                   : vanka_build_dim<T, 3>(lv, pb, U, vstar, EA, EB, EM, inv, invh, scale, status, work, s);
}

template <typename T>
cudaError_t vanka_apply(const Level& lv, const Problem& pb, const T* inv, const void* invh, const float* scale,
                        const T* res, T* d, double omega, double omega_p, int color, int* wstat, cudaStream_t s,
                        unsigned extra_tx, int slots) {
  return lv.d == 2 ? vanka_apply_dim<T, 2>(lv, pb, inv, invh, scale, res, d, omega, omega_p, color, wstat, s, extra_tx, slots)
                   : vanka_apply_dim<T, 3>(lv, pb, inv, invh, scale, res, d, omega, omega_p, color, wstat, s, extra_tx, slots);
}

template cudaError_t vanka_build<float>(const Level&, const Problem&, const float*, float*, float*, float*, float*,
                                        float*, void*, float*, int*, float*, cudaStream_t);
template cudaError_t vanka_build<double>(const Level&, const Problem&, const double*, double*, double*, double*,
                                         double*, double*, void*, float*, int*, double*, cudaStream_t);
template cudaError_t vanka_apply<float>(const Level&, const Problem&, const float*, const void*, const float*,
                                        const float*, float*, double, double, int, int*, cudaStream_t, unsigned, int);
template cudaError_t vanka_apply<double>(const Level&, const Problem&, const double*, const void*, const float*,
                                         const double*, double*, double, double, int, int*, cudaStream_t, unsigned, int);

}  // namespace stmg
