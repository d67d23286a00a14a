// Vanka launch templates shared by the per-dimension translation units (vanka_d2_*.cu,
// vanka_d3_*.cu) and the dispatch in vanka.cu: shared-memory budgets, the build of one level and
// the colour launches of one sweep, per element type T, dimension D and N = r + 2.
#pragma once
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "mg.hpp"
#include "op_launch.cuh"
#include "vanka.cuh"
#include "vanka_diag.cuh"
#include "vanka_exact.cuh"
#include "vec.cuh"
#include "counters.hpp"

namespace stmg {




template <int D, int N>
static size_t elem_smem(size_t es) {
  constexpr int Q = Shape<D, N>::Q, NL = Q, NF = Shape<D, N>::NF;
  constexpr int FSZ = NF * (2 + 2 * D) + 2 * NF * NL;
  return es * (Q * NL * D + Q * NL + Q + Q * D + D * NL + D * FSZ + 8 + 24);
}

static size_t patch_smem(const Level& lv, size_t es) {
  const size_t ms = vanka_spatial_size(lv);
  size_t nl = 1;
  for (int l = 0; l < lv.d; ++l) nl *= (lv.r + 2);
  const size_t mv = lv.d * nl;
  return es * (2 * ms * ms + mv * mv + nl * nl + 2 * ms) + sizeof(int) * ms + 16;
}

static size_t elem_smem_any(const Level& lv, size_t es) {
  int N = lv.r + 2;
  if (lv.d == 2) return N == 3 ? elem_smem<2, 3>(es) : N == 4 ? elem_smem<2, 4>(es) : elem_smem<2, 5>(es);
  return N == 3 ? elem_smem<3, 3>(es) : N == 4 ? elem_smem<3, 4>(es) : elem_smem<3, 5>(es);
}

// The patch matrices of a cell fit shared memory (else k_patch_global, global workspace).
static bool patch_onchip(const Level& lv, size_t es) { return patch_smem(lv, es) <= 227 * 1024; }

// Consumer groups of the warp-specialised persistent apply (k_vanka_apply_ws), which serves 2D
// patches of more than 32 rows: 5 by default (at most half the stages); the environment variable
// STMG_VANKA_WS overrides it (0: one-shot k_vanka_apply blocks, kept for comparisons; read once).
inline int vanka_ws_groups() {
  static const int c = [] {
    const char* v = std::getenv("STMG_VANKA_WS");
    if (!v) return 5;
    const int x = std::atoi(v);
    return x < 0 ? 0 : (x > 8 ? 8 : x);
  }();
  return c;
}
inline bool vanka_ws_enabled() { return vanka_ws_groups() > 0; }

// The stored inverse blob of a cell fits shared memory (else k_vanka_apply_global).
static bool apply_onchip(const Level& lv, size_t es_store, size_t es) {
  return apply_slot_bytes(lv.k + 1, (int)vanka_spatial_size(lv), es_store, es) <= 227 * 1024;
}

// Shared memory of k_patch_diag: inverse temporal blocks, Schur complement, pivots, column.
static size_t patch_diag_smem(const Level& lv, size_t es) {
  const size_t mv = vanka_spatial_size(lv) - lv.npc, kp1 = lv.k + 1, ns = kp1 * lv.npc;
  return es * (mv * kp1 * kp1 + ns * ns + 2 * ns + 2) + sizeof(int) * (ns + 1);
}

// The per-cell tables of the element-matrix kernel fit shared memory (else k_elem_global).
static bool elem_onchip(const Level& lv, size_t es) { return elem_smem_any(lv, es) <= 227 * 1024; }

static size_t elem_table_any(const Level& lv) {
  int N = lv.r + 2;
  if (lv.d == 2) return N == 3 ? elem_table_entries<2, 3>() : N == 4 ? elem_table_entries<2, 4>() : elem_table_entries<2, 5>();
  return N == 3 ? elem_table_entries<3, 3>() : N == 4 ? elem_table_entries<3, 4>() : elem_table_entries<3, 5>();
}


// Block slots of the global build workspace and their size in entries.
constexpr int kWorkSlots = 152 * 2;
static size_t work_slot(const Level& lv) {
  const size_t ms = vanka_spatial_size(lv);
  size_t nl = 1;
  for (int l = 0; l < lv.d; ++l) nl *= (lv.r + 2);
  const size_t mv = lv.d * nl;
  return 2 * ms * ms + mv * mv + nl * nl;
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
                            T* inv, void* invh, float* scale, int* status, T* work, cudaStream_t s) {
  Tab<T> tb = make_tab<T>(lv.tabs, pb.tau);
  int64_t ncells = lv.Np / lv.npc;
  int64_t g = (lv.Nv + 255) / 256; if (g > 152 * 8) g = 152 * 8;
  k_midpoint<T><<<(int)g, 256, 0, s>>>(U, vstar, lv.Nv, lv.k + 1, tb);
  const bool diag = lv.smoother == 1;
  const bool onchip = diag || patch_onchip(lv, sizeof(T));
  const bool eon = elem_onchip(lv, sizeof(T));
  if ((!onchip || !eon) && !work) return cudaErrorInvalidValue;
  VankaArgs<T> V{level_args<T>(lv, pb, 0.0), vstar, EA, EB, EM, 0, inv, (__half*)invh, scale, status,
                 onchip ? nullptr : work, onchip ? 0 : (int64_t)work_slot(lv)};
  size_t es = elem_smem<D, N>(sizeof(T));
  cudaError_t e = cudaSuccess;
  if (eon) {
    e = allow_smem(k_elem<T, D, N>, es);
    if (e != cudaSuccess) return e;
  }
  size_t ps = 0;
  if (lv.smoother == 2) {
    const int ms = (int)vanka_spatial_size(lv), mv = ms - lv.npc;
    ps = patch_exact_smem((lv.k + 1) * ms, mv, mv / D, sizeof(T));
    e = allow_smem(k_patch_exact<T, D, N>, ps);
    if (e != cudaSuccess) return e;
  } else if (diag) {
    ps = patch_diag_smem(lv, sizeof(T));
    e = allow_smem(k_patch_diag<T, D, N>, ps);
    if (e != cudaSuccess) return e;
  } else if (onchip) {
    ps = patch_smem(lv, sizeof(T));
    e = allow_smem(k_patch<T, D, N>, ps);
    if (e != cudaSuccess) return e;
  } else {
    const size_t ms = vanka_spatial_size(lv);
    ps = sizeof(T) * 2 * ms + sizeof(int) * ms + 16;
  }
  const TEig<T> te = make_teig<T>(lv.tabs, pb.tau);
  // chunks of whole cell planes (the last coordinate): the element matrices of the chunk and of
  // one plane on either side (the patches' neighbours) fit the scratch of vanka_elem_cells cells
  const int64_t plane = ncells / lv.n;
  int64_t planes = (int64_t)vanka_elem_cells(lv) >= ncells ? lv.n : (int64_t)vanka_elem_cells(lv) / plane - 2;
  if (planes < 1 || planes > lv.n) planes = lv.n;
  for (int64_t z0 = 0; z0 < lv.n; z0 += planes) {
    const int64_t z1 = z0 + planes < lv.n ? z0 + planes : lv.n;
    const int64_t e0 = (z0 > 0 ? z0 - 1 : 0) * plane, e1 = (z1 < lv.n ? z1 + 1 : lv.n) * plane;
    const int64_t p0 = z0 * plane, p1 = z1 * plane;
    V.ebase = e0;
    if (lv.smoother == 2) {
      // exact patches: velocity element blocks at every time node's own state (the level state,
      // velocity part V^a at U + a N_v)
      const int64_t stride = (int64_t)vanka_elem_cells(lv) * (int64_t)vanka_elem_size(lv, 0);
      for (int a = 0; a <= lv.k; ++a) {
        VankaArgs<T> Va = V;
        Va.vstar = U + (int64_t)a * lv.Nv;
        Va.EA = EA + a * stride;
        k_elem<T, D, N><<<(unsigned)(e1 - e0), 256, es, s>>>(Va, tb, e0, e1);
      }
      k_patch_exact<T, D, N><<<(unsigned)(p1 - p0), 256, ps, s>>>(V, tb, stride, p0, p1);
      note_launch(lv.k + 2);
      continue;
    }
    if (eon) {
      k_elem<T, D, N><<<(unsigned)(e1 - e0), 256, es, s>>>(V, tb, e0, e1);
    } else {
      // tables in global memory: one slot per block (the slots precede any patch workspace use,
      // which follows on the same stream)
      VankaArgs<T> Ve = V;
      Ve.work = work;
      const int64_t grid = e1 - e0 < kWorkSlots ? e1 - e0 : kWorkSlots;
      k_elem_global<T, D, N><<<(unsigned)grid, 256, 0, s>>>(Ve, tb, e0, e1);
    }
    if (diag) {
      k_patch_diag<T, D, N><<<(unsigned)(p1 - p0), 128, ps, s>>>(V, tb, p0, p1);
    } else if (onchip) {
      // 3D patches (m_s = 85 for Q2/P1): more threads shorten each elimination step
      k_patch<T, D, N><<<(unsigned)(p1 - p0), D == 3 ? 512 : 256, ps, s>>>(V, tb, te, p0, p1);
    } else {
      const int64_t grid = p1 - p0 < kWorkSlots ? p1 - p0 : kWorkSlots;
      k_patch_global<T, D, N><<<(unsigned)grid, 512, ps, s>>>(V, tb, te, p0, p1);
    }
    note_launch(2);
  }
  note_launch(1);
  return cudaGetLastError();
}

template <typename T, typename SI, int D, int N>
static cudaError_t apply_cells(const Level& lv, const Problem& pb, const SI* inv, const float* scale, const T* res,
                               T* d, double omega, double omega_p, const ColorInfo& ci, int* wstat,
                               unsigned extra_tx, cudaStream_t s, int slots, SlotStrides zs) {
  // one block per cell, threads = spatial patch rows rounded up to whole warps
  const int ms = (int)vanka_spatial_size(lv), kp1 = lv.k + 1;
  if (ms != patch_rows<D, N>()) return cudaErrorInvalidValue;
  const int threads = ((ms + 31) / 32) * 32;
  if (!apply_onchip(lv, sizeof(SI), sizeof(T))) {
    const int mr = (ms + 1) & ~1;
    const size_t gsm = (((size_t)kp1 * mr * sizeof(T) + 7) & ~(size_t)7) + (size_t)ms * 8;
    k_vanka_apply_global<T, SI, D, N><<<dim3((unsigned)ci.count, slots), threads, gsm, s>>>(
        level_args<T>(lv, pb, 0.0), inv, scale, res, d, (T)omega, (T)omega_p, kp1, lv.npc,
        make_teig<T>(lv.tabs, pb.tau), ci, zs);
    return cudaSuccess;
  }
  // 2D patches of more than one warp's rows: the warp-specialised persistent kernel, one block
  // per SM, as many stages as fit 200 KB of shared memory
  if constexpr (D == 2) {
    if (threads > 32 && vanka_ws_enabled()) {
      const size_t blob = apply_blob_bytes(kp1, ms, sizeof(SI));
      const size_t rtb = ws_rt_bytes(kp1, ms, sizeof(T));
      const int cw = vanka_ws_groups();
      int S = (int)((200 * 1024 - cw * rtb - 16) / (blob + 16));
      if (S > 16) S = 16;
      int C = S >= 2 * cw ? cw : S / 2;
      // the block's registers must fit the SM's 64 K
      cudaFuncAttributes fa{};
      cudaError_t e = cudaFuncGetAttributes(&fa, k_vanka_apply_ws<T, SI, D, N>);
      if (e != cudaSuccess) return e;
      const int regs = (fa.numRegs + 7) & ~7;        // allocation granularity
      while (C > 1 && ((32 + C * threads) * regs > 65536 || 32 + C * threads > fa.maxThreadsPerBlock)) --C;
      if (C >= 1 && (32 + C * threads) * regs <= 65536 && 32 + C * threads <= fa.maxThreadsPerBlock) {
        const size_t wsm = ws_smem_bytes(kp1, ms, sizeof(SI), sizeof(T), S, C);
        e = allow_smem(k_vanka_apply_ws<T, SI, D, N>, wsm);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const unsigned grid = (unsigned)(ci.count < sms ? ci.count : sms);
        k_vanka_apply_ws<T, SI, D, N><<<dim3(grid, slots), 32 + C * threads, wsm, s>>>(
            level_args<T>(lv, pb, 0.0), inv, scale, res, d, (T)omega, (T)omega_p, kp1, lv.npc,
            make_teig<T>(lv.tabs, pb.tau), ci, wstat, extra_tx, zs, S, C, threads);
        return cudaSuccess;
      }
    }
  }
  // cells per block: 4 for one-warp patches (32 resident blocks per SM), else 1
  const size_t slot = apply_slot_bytes(kp1, ms, sizeof(SI), sizeof(T));
  int cpb = threads <= 32 ? 4 : 1;
  while (cpb > 1 && (size_t)cpb * slot > 100 * 1024) cpb /= 2;
  const size_t smem = (size_t)cpb * slot;
  cudaError_t e = allow_smem(k_vanka_apply<T, SI, D, N>, smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((ci.count + cpb - 1) / cpb);
  k_vanka_apply<T, SI, D, N><<<dim3(blocks, slots), threads * cpb, smem, s>>>(
      level_args<T>(lv, pb, 0.0), inv, scale, res, d, (T)omega, (T)omega_p, kp1, lv.npc,
      make_teig<T>(lv.tabs, pb.tau), ci, wstat, extra_tx, zs);
  return cudaSuccess;
}

template <typename T, int D, int N>
static cudaError_t apply_dn(const Level& lv, const Problem& pb, const T* inv, const void* invh, const float* scale,
                            const T* res, T* d, double omega, double omega_p, int color, int* wstat,
                            unsigned extra_tx, cudaStream_t s, int slots) {
  const ColorInfo& ci = lv.colors[color];
  if (ci.count == 0) return cudaSuccess;
  const int64_t cells = lv.Np / lv.npc;
  const SlotStrides zs{cells * (int64_t)vanka_inv_entries(lv, invh ? 2 : (int)sizeof(T)), cells * (lv.k + 1),
                       lv.Nst};
  if (lv.smoother == 2) {
    const int ms = (int)vanka_spatial_size(lv), mst = (lv.k + 1) * ms;
    const size_t smem = apply_exact_smem(mst, ms, sizeof(T));
    cudaError_t e = allow_smem(k_vanka_apply_exact<T, D, N>, smem);
    if (e != cudaSuccess) return e;
    k_vanka_apply_exact<T, D, N><<<dim3((unsigned)ci.count, slots), ((mst + 31) / 32) * 32, smem, s>>>(
        level_args<T>(lv, pb, 0.0), inv, res, d, (T)omega, (T)omega_p, lv.k + 1, lv.npc, ci, wstat, extra_tx, zs);
    note_launch();
    return cudaGetLastError();
  }
  if (lv.smoother == 1) {
    // diagonal space-time Vanka: one warp per cell, up to four cells per block
    constexpr int NL = Shape<D, N>::Q;
    const size_t slot = diag_slot_bytes(D * NL, lv.npc, lv.k + 1, sizeof(T));
    int cpb = 4;
    while (cpb > 1 && (size_t)cpb * slot > 200 * 1024) --cpb;
    const size_t smem = (size_t)cpb * slot;
    cudaError_t e = allow_smem(k_vanka_apply_diag<T, D, N>, smem);
    if (e != cudaSuccess) return e;
    k_vanka_apply_diag<T, D, N><<<dim3((unsigned)((ci.count + cpb - 1) / cpb), slots), 32 * cpb, smem, s>>>(
        level_args<T>(lv, pb, 0.0), inv, res, d, (T)omega, (T)omega_p, make_tab<T>(lv.tabs, pb.tau), ci, cpb, zs);
    note_launch();
    return cudaGetLastError();
  }
  cudaError_t e = invh ? apply_cells<T, __half, D, N>(lv, pb, (const __half*)invh, scale, res, d, omega, omega_p, ci,
                                                      wstat, extra_tx, s, slots, zs)
                       : apply_cells<T, T, D, N>(lv, pb, inv, nullptr, res, d, omega, omega_p, ci, wstat, extra_tx,
                                                 s, slots, zs);
  if (e != cudaSuccess) return e;
  note_launch();
  return cudaGetLastError();
}


// Dispatch on N for one (T, D), instantiated in the per-dimension translation units.
template <typename T, int D>
cudaError_t vanka_build_dim(const Level& lv, const Problem& pb, const T* U, T* vstar, T* EA, T* EB, T* EM,
                            T* inv, void* invh, float* scale, int* status, T* work, cudaStream_t s) {
  const int N = lv.r + 2;
  if (N == 3) return build_dn<T, D, 3>(lv, pb, U, vstar, EA, EB, EM, inv, invh, scale, status, work, s);
  if (N == 4) return build_dn<T, D, 4>(lv, pb, U, vstar, EA, EB, EM, inv, invh, scale, status, work, s);
  if (N == 5) return build_dn<T, D, 5>(lv, pb, U, vstar, EA, EB, EM, inv, invh, scale, status, work, s);
  return cudaErrorNotSupported;
}

template <typename T, int D>
cudaError_t vanka_apply_dim(const Level& lv, const Problem& pb, const T* inv, const void* invh, const float* scale,
                            const T* res, T* d, double omega, double omega_p, int color, int* wstat, cudaStream_t s,
                            unsigned extra_tx, int slots) {
  const int N = lv.r + 2;
  if (N == 3) return apply_dn<T, D, 3>(lv, pb, inv, invh, scale, res, d, omega, omega_p, color, wstat, extra_tx, s, slots);
  if (N == 4) return apply_dn<T, D, 4>(lv, pb, inv, invh, scale, res, d, omega, omega_p, color, wstat, extra_tx, s, slots);
  if (N == 5) return apply_dn<T, D, 5>(lv, pb, inv, invh, scale, res, d, omega, omega_p, color, wstat, extra_tx, s, slots);
  return cudaErrorNotSupported;
}

}  // namespace stmg
