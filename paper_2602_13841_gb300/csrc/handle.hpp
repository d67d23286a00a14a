// The opaque handle behind stmg_handle: parameters, stream, levels, multigrid, Krylov and
// Newton work space, phase timers.
#pragma once
#include <stdexcept>
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/stmg.h"
#include "level.hpp"
#include "mg.hpp"

namespace stmg {

// Kernel classes of the profile: FP64 Jacobian apply, preconditioner-precision Jacobian apply,
// residual, Vanka patch apply (one launch per colour), Vanka build, mass apply.
enum KernelClass { KC_APPLY64 = 0, KC_APPLYP = 1, KC_RESIDUAL = 2, KC_VANKA_APPLY = 3, KC_VANKA_BUILD = 4,
                   KC_MASS = 5, KC_VANKA_APPLY0 = 6, KC_COUNT = 7 };

// Accumulates device time of one phase from CUDA event pairs recorded on the handle's stream.
struct PhaseTimer {
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spans;
  size_t used = 0;
  double ms = 0.0;
  cudaEvent_t get();
  void begin(cudaStream_t s);
  void end(cudaStream_t s);
  void collect();            // after a stream synchronisation: add the spans to ms
  ~PhaseTimer();
  cudaEvent_t open_ = nullptr;
};

struct CudaFailure : std::runtime_error {
  cudaError_t err;
  explicit CudaFailure(cudaError_t e) : std::runtime_error(cudaGetErrorString(e)), err(e) {}
};

struct Handle {
  stmg_params prm{};
  cudaStream_t stream = nullptr;
  int device = 0;                     // the CUDA device that was current at stmg_create
  Problem pb{};
  std::vector<Level> levels;
  std::vector<void*> allocs;
  std::string err;
  // preconditioner (one of the two, by prm.precond_precision)
  std::unique_ptr<MG<float>> mg32;
  std::unique_ptr<MG<double>> mg64;
  // outer FP64 work space (level 0)
  double *Vb = nullptr, *Zb = nullptr, *w = nullptr, *R = nullptr, *dX = nullptr, *Xt = nullptr;
  double *Mv = nullptr, *Jv = nullptr, *pw = nullptr, *scratch = nullptr, *hdev = nullptr;
  int* flag = nullptr;
  // STMG_USER data: host callbacks, their evaluation points on the finest level (SoA), device
  // tables of f and g for the slab starting at user_t0 (see LevelArgs::ftab / gtab)
  stmg_field_fn user_f = nullptr, user_g = nullptr;
  void* user_ctx = nullptr;
  std::vector<double> user_fx, user_gx;
  double* ftab = nullptr;
  double* gtab = nullptr;
  double user_t0 = 0.0;
  bool user_valid = false;
  std::vector<double> verts0;         // host copy of the finest level's vertices
  bool solver_ready = false;
  // batched preconditioning: the group this handle is attached to and its slot there
  struct Group* group = nullptr;
  int slot = -1;
  bool timing = false;
  bool wait_fault = false;           // failure-test hook: Vanka applies wait for bytes never sent
  PhaseTimer t_rebuild, t_mg;
  // per kernel class (KernelClass) device time, launch count and algorithmic bytes, timing mode
  PhaseTimer kt[8];
  long long kcount[8] = {};
  double kbytes[8] = {};
  // While a CUDA graph is being captured, timer spans get their own events (graph event-record
  // nodes) and go to `capsink`; they are read after every replay of that graph.
  std::vector<CapSpan>* capsink = nullptr;
  cudaEvent_t cap_open[8] = {};
  unsigned kmask = ~0u;               // kernel classes that record timer spans
  bool ktimed(int cls) const { return timing && ((kmask >> cls) & 1u); }
  void kbegin(int cls) {
    if (!ktimed(cls)) return;
    // external event-record nodes: the graph records these events at every replay
    if (capsink) { cudaEventCreate(&cap_open[cls]); cudaEventRecordWithFlags(cap_open[cls], stream, cudaEventRecordExternal); }
    else kt[cls].begin(stream);
  }
  void kend(int cls, double bytes = 0.0, int launches = 1) {
    if (!ktimed(cls)) return;
    if (capsink) {
      cudaEvent_t e; cudaEventCreate(&e); cudaEventRecordWithFlags(e, stream, cudaEventRecordExternal);
      capsink->push_back({cls, cap_open[cls], e, bytes, launches});
    } else { kt[cls].end(stream); kcount[cls] += launches; kbytes[cls] += bytes; }
  }
  ~Handle();
  void* dalloc(size_t bytes);          // cudaMalloc tracked for release; throws std::bad_alloc
  // host -> device copy of set-up data on the handle's stream, complete on return (the host
  // buffer may be freed right after); throws CudaFailure.  No device-wide or legacy-stream
  // synchronisation: other handles may be capturing graphs on their streams meanwhile.
  void upload(void* dst, const void* src, size_t bytes);
  stmg_status fail(stmg_status s, const std::string& msg);
  cudaError_t ensure_mg();
  cudaError_t ensure_solver();
  bool precond_fp32() const { return prm.precond_precision == STMG_FP32; }
};

}  // namespace stmg
