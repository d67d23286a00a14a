// Vanka smoother sweep that allocates nothing: the residual scratch lives in a file-scope device
// array instead of the handle's level work vector.  See stmg_smoother_sweep_noalloc in stmg.h.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/stmg.h"
#include "handle.hpp"
#include "vec.cuh"

namespace stmg {

// 4 MiB, held by every GPU that loads this library until the process exits.
constexpr int64_t kNoallocScratchBytes = (int64_t)1 << 22;
static __device__ __align__(256) double g_sweep_scratch[kNoallocScratchBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices] = {};
static std::mutex g_scratch_mutex;

// Device address of g_sweep_scratch on the current device (looked up once per device; the host
// symbol itself is only a stand-in and must never be passed to a kernel).
static cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sweep_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

template <typename T>
static cudaError_t sweep_noalloc(Handle* h, MG<T>& mg, int l, const T* rhs, T* d, int nsweeps, bool zero_start,
                                 T* q) {
  cudaStream_t s = h->stream;
  const Level& lv = h->levels[l];
  for (int it = 0; it < nsweeps; ++it) {
    const T* res = rhs;
    if (it == 0 && zero_start) {
      cudaError_t e = cudaMemsetAsync(d, 0, lv.Nst * sizeof(T), s);
      if (e != cudaSuccess) return e;
    } else {
      // q = rhs - J d, by the same launches as the regular sweep
      cudaError_t e = launch_level_residual<T>(lv, h->pb, rhs, d, mg.U[l], q, s);
      if (e != cudaSuccess) return e;
      res = q;
    }
    for (int c = 0; c < lv.ncolors; ++c) {
      cudaError_t e = vanka_apply<T>(lv, h->pb, mg.inv[l], mg.invh[l], mg.iscale[l], res, d, h->prm.omega,
                                     h->prm.omega_p, c, mg.wstat, s, h->wait_fault ? 16u : 0u);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace stmg

using namespace stmg;

extern "C" stmg_status stmg_smoother_sweep_noalloc(stmg_handle* hh, int level, const void* rhs, void* d,
                                                   int nsweeps, int zero_start) {
  if (!hh || !rhs || !d || nsweeps < 0) return STMG_ERR_ARG;
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (level < 0 || level + 1 >= (int)h->levels.size())
    return h->fail(STMG_ERR_ARG, "smoother_sweep_noalloc: level has no smoother");
  const bool fp32 = h->precond_fp32();
  const bool built = fp32 ? (h->mg32 && h->mg32->built) : (h->mg64 && h->mg64->built);
  if (!built) return h->fail(STMG_ERR_ARG, "smoother_sweep_noalloc: call stmg_smoother_build first");
  const int64_t esize = fp32 ? (int64_t)sizeof(float) : (int64_t)sizeof(double);
  const int64_t need = h->levels[level].Nst * esize;
  if (need > kNoallocScratchBytes)
    return h->fail(STMG_ERR_ARG, "smoother_sweep_noalloc: level vector of " + std::to_string(need) +
                                     " bytes exceeds the fixed scratch of " + std::to_string(kNoallocScratchBytes) +
                                     " bytes");
  // the array's address is per device: look it up on the device the handle's stream belongs to
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != h->device) {
    cudaGetLastError();
    return h->fail(STMG_ERR_ARG, "smoother_sweep_noalloc: the current CUDA device (" + std::to_string(cur) +
                                     ") is not the device the handle was created on (" +
                                     std::to_string(h->device) + ")");
  }
  void* q = nullptr;
  cudaError_t e = scratch_address(&q);
  if (e != cudaSuccess)
    return h->fail(STMG_ERR_CUDA, std::string("smoother_sweep_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  e = fp32 ? sweep_noalloc<float>(h, *h->mg32, level, (const float*)rhs, (float*)d, nsweeps, zero_start != 0, (float*)q)
           : sweep_noalloc<double>(h, *h->mg64, level, (const double*)rhs, (double*)d, nsweeps, zero_start != 0,
                                   (double*)q);
  if (e == cudaSuccess) e = fp32 ? h->mg32->check_wait() : h->mg64->check_wait();
  if (e == cudaErrorTimeout)
    return h->fail(STMG_ERR_TIMEOUT, "smoother_sweep_noalloc: a bounded wait in the Vanka apply ran out");
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("smoother_sweep_noalloc: ") + cudaGetErrorString(e));
  return STMG_OK;
}
