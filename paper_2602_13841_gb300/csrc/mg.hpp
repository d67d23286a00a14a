// hp space-time multigrid preconditioner (Sec. 4.2-4.3) on the device, element type T of the
// preconditioner (float: mixed precision; double: plain FP64).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "level.hpp"
#include "transfer.hpp"

namespace stmg {

struct Handle;

// A timer span (kernel class, begin / end events, algorithmic bytes, launches) recorded inside
// a captured CUDA graph.
struct CapSpan { int cls; cudaEvent_t a, b; double bytes; int launches; };

template <typename T>
struct MG {
  Handle* h = nullptr;
  int nl = 0;
  // Slots: B independent solves of the same level shapes share this hierarchy and are carried
  // through one V-cycle by the same launches (slot j's vectors at j * n_st of each level, its patch
  // inverses and coarse factors at slot strides); nub holds each slot's viscosity (device, B > 1).
  int B = 1;
  T* nub = nullptr;
  std::vector<int64_t> inv_slot, invh_slot, scale_slot;   // per level: slot strides of the patch data
  std::vector<T*> U, r, z, t, q;     // per level: state, rhs, correction, temporaries
  std::vector<T*> inv;               // per smoothed level: patch inverses (precision T) ...
  std::vector<void*> invh;           // ... or FP16 patch inverses (params.vanka_fp16) ...
  std::vector<float*> iscale;        // ... with one FP32 scale per patch
  std::vector<Transfer> tr;
  T *EA = nullptr, *EB = nullptr, *EM = nullptr, *vstar = nullptr;
  T* work = nullptr;                 // global workspace of the large-patch build
  int* status = nullptr;             // device flag: zero pivot in a patch
  int* wstat = nullptr;              // device flag: a bounded wait in the Vanka apply ran out
  cudaError_t check_wait();          // reads and clears wstat (synchronises the stream)
  // coarsest level: bordered Jacobian (FP64), its FP64 inverse, refinement buffers
  int Nc = 0, Nb = 0;
  double *A64 = nullptr, *Ucs = nullptr, *cb = nullptr, *cx = nullptr, *cr = nullptr, *cw = nullptr;
  double* ident = nullptr;
  double* Ainv = nullptr;
  double* gj_col = nullptr;
  int* gj_piv = nullptr;
  bool built = false;
  bool smoothable = true;            // every smoothed level's element matrices fit on-chip memory
  // The V-cycle of one smoother build is a fixed launch sequence on fixed buffers: it is
  // captured once into a CUDA graph and replayed (launch overhead of the ~40 small launches per
  // level).  Timer spans recorded during the capture are re-read after every replay.
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_slots = 1;               // slots the captured graph covers
  bool use_graph = true;
  bool graph_timing = false;         // the captured graph contains timer event nodes ...
  unsigned graph_kmask = ~0u;        // ... of these kernel classes
  int graph_kernels = 0;             // kernel launches recorded in the graph (counted per replay)
  std::vector<CapSpan> gspans;       // timer spans inside the captured graph
  void drop_graph();
  cudaError_t vcycle_graph(int slots = 1);   // z[0] = B^{-1} r[0] through the captured graph
  void collect_graph_timers();       // after a stream synchronisation following a replay

  cudaError_t allocate(Handle* h, int slots = 1);
  // Level states from the fine FP64 slab state, patch inverses on every smoothed level,
  // coarse factorisation, for one slot (physics pb; the handle's when null).  Returns
  // cudaErrorUnknown if a patch has a zero pivot.
  cudaError_t setup(const double* U64, int slot = 0, const Problem* pb = nullptr);
  // z = B^{-1} rhs on level 0 (rhs, z: level-0 vectors of type T), for the first `slots` slots
  // (0: all B).
  cudaError_t vcycle(const T* rhs, T* z, int slots = 0);
  cudaError_t vcycle_level(int l, const T* rhs, T* d, int slots);
  // nsweeps Vanka sweeps on level l: d <- d + omega sum_K ... (rhs - J d); `zero_start`: d = 0 on entry.
  cudaError_t sweep(int l, const T* rhs, T* d, int nsweeps, bool zero_start, int slots = 1);
  cudaError_t coarse_solve(const T* rhs, T* d, int slots = 1);
};

// Launch helpers implemented in vanka.cu (templated on T).
template <typename T>
cudaError_t vanka_build(const Level& lv, const Problem& pb, const T* U, T* vstar, T* EA, T* EB, T* EM,
                        T* inv, void* invh, float* scale, int* status, T* work, cudaStream_t s);
size_t vanka_work_entries(const Level& lv, size_t esize);  // global build workspace (0: on-chip patches)
size_t vanka_elem_cells(const Level& lv);   // cells per chunk of the element-matrix scratch
// inv: patch inverses of precision T, or (invh non-null) FP16 inverses scaled by scale[cell].
template <typename T>
cudaError_t vanka_apply(const Level& lv, const Problem& pb, const T* inv, const void* invh, const float* scale,
                        const T* res, T* d, double omega, double omega_p, int color, int* wstat, cudaStream_t s,
                        unsigned extra_tx = 0,    // extra_tx: failure-test hook (see stmg_test_wait_timeout)
                        int slots = 1);           // independent slots: inverses, res and d at slot strides
size_t vanka_spatial_size(const Level& lv);          // m_s = d (r+2)^d + npc
size_t vanka_patch_size(const Level& lv);            // m_st = (k+1) m_s
size_t vanka_inv_entries(const Level& lv, int es);   // stored reals of one cell's patch inverse ((k+1) m_s x stride), es-byte entries
size_t vanka_elem_size(const Level& lv, int which);  // entries per cell of EA (0), EB (1), EM (2)
bool vanka_supported(const Level& lv, size_t esize);

// Coarse solver helpers (coarse.cu)
cudaError_t coarse_border(const Level& lv, const Problem& pb, const double* J, double* A, int N, int Nb,
                          cudaStream_t s);
cudaError_t coarse_invert(const double* A, double* Ainv, double* col, int* piv, int Nb, int* status,
                          cudaStream_t s);
// y_j = A_j x_j for j < slots (A_j = A + j n^2, x_j = x + j n, y_j = y + j n); column-major.
cudaError_t gemv_cm(const double* A, int n, const double* x, double* y, cudaStream_t s, int slots = 1);

}  // namespace stmg
