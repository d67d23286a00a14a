// hp-STMG V-cycle on the device (Sec. 4.2): p-coarsening first, then h; nu1 / nu2 Vanka sweeps;
// restriction = transpose of the prolongation; coarsest level solved directly.
#include <type_traits>

#include "handle.hpp"
#include "mg.hpp"
#include "vec.cuh"
#include "counters.hpp"

namespace stmg {

#define CKE(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return e_; } while (0)

template <typename T>
cudaError_t MG<T>::allocate(Handle* hh) {
  h = hh;
  nl = (int)h->levels.size();
  U.resize(nl); r.resize(nl); z.resize(nl); t.resize(nl); q.resize(nl); inv.assign(nl, nullptr);
  invh.assign(nl, nullptr); iscale.assign(nl, nullptr);
  size_t ea = 0, eb = 0, em = 0, nv = 0, wk = 0;
  try {
    for (int l = 0; l < nl; ++l) {
      const Level& lv = h->levels[l];
      U[l] = (T*)h->dalloc(lv.Nst * sizeof(T));
      r[l] = (T*)h->dalloc(lv.Nst * sizeof(T));
      z[l] = (T*)h->dalloc(lv.Nst * sizeof(T));
      t[l] = (T*)h->dalloc(lv.Nst * sizeof(T));
      q[l] = (T*)h->dalloc(lv.Nst * sizeof(T));
      if (l < nl - 1) {
        if (!vanka_supported(lv, sizeof(T))) { smoothable = false; continue; }
        size_t m = vanka_patch_size(lv);
        if (h->prm.vanka_fp16 && lv.smoother == 0) {
          invh[l] = h->dalloc((size_t)(lv.Np / lv.npc) * vanka_inv_entries(lv, 2) * 2);
          iscale[l] = (float*)h->dalloc((size_t)(lv.Np / lv.npc) * (lv.k + 1) * sizeof(float));
        } else {
          inv[l] = (T*)h->dalloc((size_t)(lv.Np / lv.npc) * vanka_inv_entries(lv, (int)sizeof(T)) * sizeof(T));
        }
        size_t nc = lv.Np / lv.npc;
        const size_t ec = vanka_elem_cells(lv);                 // element scratch: one chunk
        ea = std::max(ea, ec * vanka_elem_size(lv, 0) * (lv.smoother == 2 ? (size_t)(lv.k + 1) : 1));
        eb = std::max(eb, ec * vanka_elem_size(lv, 1));
        em = std::max(em, ec * vanka_elem_size(lv, 2));
        nv = std::max(nv, (size_t)lv.Nv);
        wk = std::max(wk, vanka_work_entries(lv, sizeof(T)));
      }
    }
    if (wk) work = (T*)h->dalloc(wk * sizeof(T));
    if (nl > 1) {
      EA = (T*)h->dalloc(ea * sizeof(T));
      EB = (T*)h->dalloc(eb * sizeof(T));
      EM = (T*)h->dalloc(em * sizeof(T));
      vstar = (T*)h->dalloc(nv * sizeof(T));
    }
    status = (int*)h->dalloc(sizeof(int));
    wstat = (int*)h->dalloc(sizeof(int));
    tr.resize(nl > 0 ? nl - 1 : 0);
    for (int l = 0; l + 1 < nl; ++l) build_transfer(h, tr[l], h->levels[l], h->levels[l + 1], sizeof(T));
    const Level& c = h->levels[nl - 1];
    Nc = (int)c.Nst;
    Nb = Nc + c.k + 1;
    A64 = (double*)h->dalloc((size_t)Nb * Nb * sizeof(double));
    ident = (double*)h->dalloc(((size_t)Nc * Nc + 2 * (size_t)Nc) * sizeof(double));
    Ucs = (double*)h->dalloc((size_t)Nc * sizeof(double));
    cb = (double*)h->dalloc((size_t)Nb * sizeof(double));
    cx = (double*)h->dalloc((size_t)Nb * sizeof(double));
    cr = (double*)h->dalloc((size_t)Nb * sizeof(double));
    cw = (double*)h->dalloc((size_t)Nb * sizeof(double));
    Ainv = (double*)h->dalloc((size_t)Nb * Nb * sizeof(double));
    gj_col = (double*)h->dalloc((size_t)Nb * sizeof(double));
    gj_piv = (int*)h->dalloc((size_t)Nb * sizeof(int));
  } catch (const std::bad_alloc&) {
    return cudaErrorMemoryAllocation;
  } catch (const CudaFailure& f) {
    return f.err;
  }
  return cudaSuccess;
}

__global__ void k_identity(double* I, int n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x)
    I[e] = ((e / n) == (e % n)) ? 1.0 : 0.0;
}

template <typename T>
cudaError_t MG<T>::check_wait() {
  int v = 0;
  CKE(cudaMemcpyAsync(&v, wstat, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CKE(cudaMemsetAsync(wstat, 0, sizeof(int), h->stream));
  CKE(cudaStreamSynchronize(h->stream));
  return v ? cudaErrorTimeout : cudaSuccess;
}

template <typename T>
cudaError_t MG<T>::setup(const double* U64) {
  cudaStream_t s = h->stream;
  const Level& f = h->levels[0];
  if (!smoothable) return cudaErrorNotSupported;
  CKE(cudaMemsetAsync(status, 0, sizeof(int), s));
  CKE(cudaMemsetAsync(wstat, 0, sizeof(int), s));
  CKE((vcopy<double, T>(f.Nst, U64, U[0], s)));
  for (int l = 0; l + 1 < nl; ++l) {
    const Level& c = h->levels[l + 1];
    CKE(cudaMemsetAsync(U[l + 1], 0, c.Nst * sizeof(T), s));
    CKE(tr[l].template interp_state<T>(U[l], U[l + 1], s));
  }
  for (int l = 0; l + 1 < nl; ++l) {
    h->kbegin(KC_VANKA_BUILD);
    CKE(vanka_build<T>(h->levels[l], h->pb, U[l], vstar, EA, EB, EM, inv[l], invh[l], iscale[l], status, work, s));
    h->kend(KC_VANKA_BUILD, 0.0, 4);
  }
  // coarse: assemble J_c at the coarse state by a batched apply to the identity
  const Level& c = h->levels[nl - 1];
  CKE((vcopy<T, double>(c.Nst, U[nl - 1], Ucs, s)));
  k_identity<<<152 * 4, 256, 0, s>>>(ident, Nc);
  note_launch();
  CKE(launch_operator<double>(c, h->pb, OP_JAC, 0.0, ident, Ucs, nullptr, A64, s, Nc, Nc, Nc));
  // A64 now holds J (N x N, column-major); move into the bordered layout via `ident` as staging
  CKE(cudaMemcpyAsync(ident, A64, (size_t)Nc * Nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CKE(coarse_border(c, h->pb, ident, A64, Nc, Nb, s));
  CKE(coarse_invert(A64, Ainv, gj_col, gj_piv, Nb, status, s));
  int st = 0;
  CKE(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaStreamSynchronize(s));
  built = true;
  return st ? cudaErrorUnknown : cudaSuccess;
}

template <typename T>
cudaError_t MG<T>::coarse_solve(const T* rhs, T* d) {
  cudaStream_t s = h->stream;
  CKE(cudaMemsetAsync(cb, 0, Nb * sizeof(double), s));
  CKE((vcopy<T, double>(Nc, rhs, cb, s)));
  CKE(gemv_cm(Ainv, Nb, cb, cx, s));
  for (int it = 0; it < 1; ++it) {          // one step of iterative refinement
    CKE(gemv_cm(A64, Nb, cx, cw, s));
    CKE(cudaMemcpyAsync(cr, cb, Nb * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CKE(vaxpby<double>(Nb, -1.0, cw, 1.0, cr, s));
    CKE(gemv_cm(Ainv, Nb, cr, cw, s));
    CKE(vaxpby<double>(Nb, 1.0, cw, 1.0, cx, s));
  }
  CKE((vcopy<double, T>(Nc, cx, d, s)));
  return cudaSuccess;
}

template <typename T>
cudaError_t MG<T>::sweep(int l, const T* rhs, T* d, int nsweeps, bool zero_start) {
  cudaStream_t s = h->stream;
  const Level& lv = h->levels[l];
  const double omega = h->prm.omega;
  for (int it = 0; it < nsweeps; ++it) {
    const T* res = rhs;
    if (it == 0 && zero_start) {
      CKE(cudaMemsetAsync(d, 0, lv.Nst * sizeof(T), s));
    } else {
      // q = rhs - J d
      h->kbegin(KC_APPLYP);
      CKE(launch_level_residual<T>(lv, h->pb, rhs, d, U[l], q[l], s));
      h->kend(KC_APPLYP);
      res = q[l];
    }
    // one timer span over the colour launches of the sweep (they run back to back);
    // algorithmic bytes: the patch inverses of every cell, residual gather, d read and write
    // per cell: (k+1) m_s^2 stored reals (one spatial inverse per real time eigenvalue, a complex
    // one per conjugate pair), residual gather and d update on the (k+1) m_s patch DoFs
    const double ms = (double)vanka_spatial_size(lv), m = (double)vanka_patch_size(lv);
    const double ib = lv.smoother != 0 ? (double)vanka_inv_entries(lv, (int)sizeof(T)) * sizeof(T)
                      : (lv.k + 1) * ms * ms * (invh[l] ? 2.0 : (double)sizeof(T)) + (invh[l] ? 4.0 * (lv.k + 1) : 0.0);
    int64_t cells = 0;
    h->kbegin(KC_VANKA_APPLY);
    if (l == 0) h->kbegin(KC_VANKA_APPLY0);
    for (int c = 0; c < lv.ncolors; ++c) {
      CKE(vanka_apply<T>(lv, h->pb, inv[l], invh[l], iscale[l], res, d, omega, h->prm.omega_p, c, wstat, s,
                         h->wait_fault ? 16u : 0u));
      cells += lv.colors[c].count;
    }
    if (l == 0) h->kend(KC_VANKA_APPLY0, (double)cells * (ib + 3.0 * m * sizeof(T)), lv.ncolors);
    h->kend(KC_VANKA_APPLY, (double)cells * (ib + 3.0 * m * sizeof(T)), lv.ncolors);
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t MG<T>::vcycle_level(int l, const T* rhs, T* d) {
  if (l == nl - 1) return coarse_solve(rhs, d);
  cudaStream_t s = h->stream;
  const Level& lv = h->levels[l];
  int nu1 = h->prm.nu1 > 0 ? h->prm.nu1 : 0, nu2 = h->prm.nu2 > 0 ? h->prm.nu2 : 0;
  // levels whose next coarser level has a lower time degree: nu_tc sweeps each way when set
  if (h->prm.nu_tc > 0 && h->levels[l + 1].k < lv.k) nu1 = nu2 = h->prm.nu_tc;
  if (nu1 > 0) CKE(sweep(l, rhs, d, nu1, true));
  else CKE(cudaMemsetAsync(d, 0, lv.Nst * sizeof(T), s));
  // t = rhs - J d ; r_{l+1} = P^T t
  h->kbegin(KC_APPLYP);
  CKE(launch_level_residual<T>(lv, h->pb, rhs, d, U[l], t[l], s));
  h->kend(KC_APPLYP);
  CKE(tr[l].template restrict_<T>(t[l], r[l + 1], s));
  CKE(vcycle_level(l + 1, r[l + 1], z[l + 1]));
  CKE(tr[l].template prolong<T>(z[l + 1], t[l], s));
  CKE(vaxpby<T>(lv.Nst, (T)1, t[l], (T)1, d, s));
  if (nu2 > 0) CKE(sweep(l, rhs, d, nu2, false));
  return cudaSuccess;
}

template <typename T>
cudaError_t MG<T>::vcycle(const T* rhs, T* zz) {
  return vcycle_level(0, rhs, zz);
}

template <typename T>
void MG<T>::drop_graph() {
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  if (graph) cudaGraphDestroy(graph);
  graph_exec = nullptr;
  graph = nullptr;
  for (auto& sp : gspans) { cudaEventDestroy(sp.a); cudaEventDestroy(sp.b); }
  gspans.clear();
}

template <typename T>
cudaError_t MG<T>::vcycle_graph() {
  cudaStream_t s = h->stream;
  if (graph_exec && (graph_timing != h->timing || graph_kmask != h->kmask)) drop_graph();
  if (!graph_exec) {
    // capture the V-cycle on r[0] -> z[0]; all buffers and parameters are fixed per handle, so
    // the graph stays valid across smoother rebuilds
    gspans.clear();
    if (h->timing) h->capsink = &gspans;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { h->capsink = nullptr; return e; }
    const long long n0 = launch_count();
    cudaError_t ev = vcycle_level(0, r[0], z[0]);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    h->capsink = nullptr;
    // kernels recorded during the capture did not run; each replay runs them all
    graph_kernels = (int)(launch_count() - n0);
    note_launch(-graph_kernels);
    if (ev != cudaSuccess) { if (g) cudaGraphDestroy(g); return ev; }
    if (e != cudaSuccess) return e;
    graph = g;
    CKE(cudaGraphInstantiate(&graph_exec, graph, 0));
    graph_timing = h->timing;
    graph_kmask = h->kmask;
  }
  CKE(cudaGraphLaunch(graph_exec, s));
  note_launch(graph_kernels);
  return cudaSuccess;
}

template <typename T>
void MG<T>::collect_graph_timers() {
  for (auto& sp : gspans) {
    float m = 0;
    if (cudaEventElapsedTime(&m, sp.a, sp.b) == cudaSuccess) {
      h->kt[sp.cls].ms += m;
      h->kcount[sp.cls] += sp.launches;
      h->kbytes[sp.cls] += sp.bytes;
    } else {
      cudaGetLastError();
    }
  }
}

template struct MG<float>;
template struct MG<double>;

}  // namespace stmg
