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
cudaError_t MG<T>::allocate(Handle* hh, int slots) {
  h = hh;
  B = slots < 1 ? 1 : slots;
  nl = (int)h->levels.size();
  U.resize(nl); r.resize(nl); z.resize(nl); t.resize(nl); q.resize(nl); inv.assign(nl, nullptr);
  invh.assign(nl, nullptr); iscale.assign(nl, nullptr);
  inv_slot.assign(nl, 0); invh_slot.assign(nl, 0); scale_slot.assign(nl, 0);
  size_t ea = 0, eb = 0, em = 0, nv = 0, wk = 0;
  try {
    if (B > 1) nub = (T*)h->dalloc(B * sizeof(T));
    for (int l = 0; l < nl; ++l) {
      const Level& lv = h->levels[l];
      U[l] = (T*)h->dalloc(B * lv.Nst * sizeof(T));
      r[l] = (T*)h->dalloc(B * lv.Nst * sizeof(T));
      z[l] = (T*)h->dalloc(B * lv.Nst * sizeof(T));
      t[l] = (T*)h->dalloc(B * lv.Nst * sizeof(T));
      q[l] = (T*)h->dalloc(B * lv.Nst * sizeof(T));
      if (l < nl - 1) {
        if (!vanka_supported(lv, sizeof(T))) { smoothable = false; continue; }
        const int64_t cells = lv.Np / lv.npc;
        if (h->prm.vanka_fp16 && lv.smoother == 0) {
          invh_slot[l] = cells * (int64_t)vanka_inv_entries(lv, 2);
          scale_slot[l] = cells * (lv.k + 1);
          invh[l] = h->dalloc((size_t)B * invh_slot[l] * 2);
          iscale[l] = (float*)h->dalloc((size_t)B * scale_slot[l] * sizeof(float));
        } else {
          inv_slot[l] = cells * (int64_t)vanka_inv_entries(lv, (int)sizeof(T));
          inv[l] = (T*)h->dalloc((size_t)B * inv_slot[l] * sizeof(T));
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
    for (int l = 0; l + 1 < nl; ++l) build_transfer(h, tr[l], h->levels[l], h->levels[l + 1], sizeof(T), B);
    const Level& c = h->levels[nl - 1];
    Nc = (int)c.Nst;
    Nb = Nc + c.k + 1;
    A64 = (double*)h->dalloc((size_t)B * Nb * Nb * sizeof(double));
    ident = (double*)h->dalloc(((size_t)Nc * Nc + 2 * (size_t)Nc) * sizeof(double));
    Ucs = (double*)h->dalloc((size_t)Nc * sizeof(double));
    cb = (double*)h->dalloc((size_t)B * Nb * sizeof(double));
    cx = (double*)h->dalloc((size_t)B * Nb * sizeof(double));
    cr = (double*)h->dalloc((size_t)B * Nb * sizeof(double));
    cw = (double*)h->dalloc((size_t)B * Nb * sizeof(double));
    Ainv = (double*)h->dalloc((size_t)B * Nb * Nb * sizeof(double));
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
cudaError_t MG<T>::setup(const double* U64, int slot, const Problem* pbp) {
  cudaStream_t s = h->stream;
  const Level& f = h->levels[0];
  const Problem& pb = pbp ? *pbp : h->pb;
  if (!smoothable) return cudaErrorNotSupported;
  if (slot < 0 || slot >= B) return cudaErrorInvalidValue;
  CKE(cudaMemsetAsync(status, 0, sizeof(int), s));
  CKE(cudaMemsetAsync(wstat, 0, sizeof(int), s));
  if (nub) {
    const T nuv = (T)pb.nu;
    CKE(cudaMemcpyAsync(nub + slot, &nuv, sizeof(T), cudaMemcpyHostToDevice, s));
  }
  auto lvec = [&](std::vector<T*>& v, int l) { return v[l] + (int64_t)slot * h->levels[l].Nst; };
  CKE((vcopy<double, T>(f.Nst, U64, lvec(U, 0), s)));
  for (int l = 0; l + 1 < nl; ++l) {
    const Level& c = h->levels[l + 1];
    CKE(cudaMemsetAsync(lvec(U, l + 1), 0, c.Nst * sizeof(T), s));
    CKE(tr[l].template interp_state<T>(lvec(U, l), lvec(U, l + 1), s));
  }
  for (int l = 0; l + 1 < nl; ++l) {
    h->kbegin(KC_VANKA_BUILD);
    CKE(vanka_build<T>(h->levels[l], pb, lvec(U, l), vstar, EA, EB, EM,
                       inv[l] ? inv[l] + slot * inv_slot[l] : nullptr,
                       invh[l] ? (void*)((unsigned short*)invh[l] + slot * invh_slot[l]) : nullptr,
                       iscale[l] ? iscale[l] + slot * scale_slot[l] : nullptr, status, work, s));
    h->kend(KC_VANKA_BUILD, 0.0, 4);
  }
  // coarse: assemble J_c at the coarse state by a batched apply to the identity
  const Level& c = h->levels[nl - 1];
  double* A64s = A64 + (int64_t)slot * Nb * Nb;
  CKE((vcopy<T, double>(c.Nst, lvec(U, nl - 1), Ucs, s)));
  k_identity<<<152 * 4, 256, 0, s>>>(ident, Nc);
  note_launch();
  CKE(launch_operator<double>(c, pb, OP_JAC, 0.0, ident, Ucs, nullptr, A64s, s, Nc, Nc, Nc));
  // A64 now holds J (N x N, column-major); move into the bordered layout via `ident` as staging
  CKE(cudaMemcpyAsync(ident, A64s, (size_t)Nc * Nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CKE(coarse_border(c, pb, ident, A64s, Nc, Nb, s));
  CKE(coarse_invert(A64s, Ainv + (int64_t)slot * Nb * Nb, gj_col, gj_piv, Nb, status, s));
  int st = 0;
  CKE(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKE(cudaStreamSynchronize(s));
  built = true;
  return st ? cudaErrorUnknown : cudaSuccess;
}

template <typename T>
cudaError_t MG<T>::coarse_solve(const T* rhs, T* d, int slots) {
  cudaStream_t s = h->stream;
  CKE(cudaMemsetAsync(cb, 0, (size_t)slots * Nb * sizeof(double), s));
  CKE((vcopy_slots<T, double>(Nc, slots, rhs, Nc, cb, Nb, s)));
  CKE(gemv_cm(Ainv, Nb, cb, cx, s, slots));
  for (int it = 0; it < 1; ++it) {          // one step of iterative refinement
    CKE(gemv_cm(A64, Nb, cx, cw, s, slots));
    CKE(cudaMemcpyAsync(cr, cb, (size_t)slots * Nb * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CKE(vaxpby<double>((int64_t)slots * Nb, -1.0, cw, 1.0, cr, s));
    CKE(gemv_cm(Ainv, Nb, cr, cw, s, slots));
    CKE(vaxpby<double>((int64_t)slots * Nb, 1.0, cw, 1.0, cx, s));
  }
  CKE((vcopy_slots<double, T>(Nc, slots, cx, Nb, d, Nc, s)));
  return cudaSuccess;
}

template <typename T>
cudaError_t MG<T>::sweep(int l, const T* rhs, T* d, int nsweeps, bool zero_start, int slots) {
  cudaStream_t s = h->stream;
  const Level& lv = h->levels[l];
  const double omega = h->prm.omega;
  for (int it = 0; it < nsweeps; ++it) {
    const T* res = rhs;
    if (it == 0 && zero_start) {
      CKE(cudaMemsetAsync(d, 0, (size_t)slots * lv.Nst * sizeof(T), s));
    } else {
      // q = rhs - J d
      h->kbegin(KC_APPLYP);
      CKE(launch_level_residual<T>(lv, h->pb, rhs, d, U[l], q[l], s, slots, slots > 1 ? nub : nullptr));
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
                         h->wait_fault ? 16u : 0u, slots));
      cells += (int64_t)slots * lv.colors[c].count;
    }
    if (l == 0) h->kend(KC_VANKA_APPLY0, (double)cells * (ib + 3.0 * m * sizeof(T)), lv.ncolors);
    h->kend(KC_VANKA_APPLY, (double)cells * (ib + 3.0 * m * sizeof(T)), lv.ncolors);
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t MG<T>::vcycle_level(int l, const T* rhs, T* d, int slots) {
  if (l == nl - 1) return coarse_solve(rhs, d, slots);
  cudaStream_t s = h->stream;
  const Level& lv = h->levels[l];
  int nu1 = h->prm.nu1 > 0 ? h->prm.nu1 : 0, nu2 = h->prm.nu2 > 0 ? h->prm.nu2 : 0;
  // levels whose next coarser level has a lower time degree: nu_tc sweeps each way when set
  if (h->prm.nu_tc > 0 && h->levels[l + 1].k < lv.k) nu1 = nu2 = h->prm.nu_tc;
  if (nu1 > 0) CKE(sweep(l, rhs, d, nu1, true, slots));
  else CKE(cudaMemsetAsync(d, 0, (size_t)slots * lv.Nst * sizeof(T), s));
  // t = rhs - J d ; r_{l+1} = P^T t
  h->kbegin(KC_APPLYP);
  CKE(launch_level_residual<T>(lv, h->pb, rhs, d, U[l], t[l], s, slots, slots > 1 ? nub : nullptr));
  h->kend(KC_APPLYP);
  CKE(tr[l].template restrict_<T>(t[l], r[l + 1], s, slots));
  CKE(vcycle_level(l + 1, r[l + 1], z[l + 1], slots));
  CKE(tr[l].template prolong<T>(z[l + 1], t[l], s, slots));
  CKE(vaxpby<T>((int64_t)slots * lv.Nst, (T)1, t[l], (T)1, d, s));
  if (nu2 > 0) CKE(sweep(l, rhs, d, nu2, false, slots));
  return cudaSuccess;
}

template <typename T>
cudaError_t MG<T>::vcycle(const T* rhs, T* zz, int slots) {
  return vcycle_level(0, rhs, zz, slots > 0 ? slots : B);
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
cudaError_t MG<T>::vcycle_graph(int slots) {
  cudaStream_t s = h->stream;
  if (graph_exec && (graph_timing != h->timing || graph_kmask != h->kmask || graph_slots != slots)) drop_graph();
  if (!graph_exec) {
    // capture the V-cycle on r[0] -> z[0]; all buffers and parameters are fixed per handle, so
    // the graph stays valid across smoother rebuilds
    gspans.clear();
    if (h->timing) h->capsink = &gspans;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { h->capsink = nullptr; return e; }
    const long long n0 = launch_count();
    cudaError_t ev = vcycle_level(0, r[0], z[0], slots);
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
    graph_slots = slots;
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
