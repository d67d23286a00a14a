// Batched preconditioning across independent slab solves of one shape (continuous batching of
// same-shape requests).  A group owns one hp-STMG hierarchy with B slots (MG<T> with B > 1):
// handles of the same shape attach to it, each to its own slot.  A handle's smoother builds fill
// its slot; its V-cycles are collected: each FGMRES iteration of an attached handle hands its
// vector to the group and waits until one batched V-cycle -- every kernel of the chain launched
// once for all ready slots (blockIdx.y / z = slot) -- has produced its correction.  A round starts
// when every handle inside a slab solve is ready, or after a short wait for the stragglers.  Slot j
// computes exactly what a lone handle computes (same kernels, per-slot data only), so a solve
// gives the same bits alone and in a batch.  All group work runs on the group's own stream
// (created here: a stream that another thread may use must never be the one a V-cycle graph is
// being captured on); the handles' streams are ordered against it with events.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/stmg.h"
#include "group.hpp"
#include "handle.hpp"
#include "vec.cuh"
#include "counters.hpp"

namespace stmg {

struct Group {
  Handle* core = nullptr;           // levels of the shape and the B-slot hierarchy (group stream)
  cudaStream_t stream = nullptr;    // owned by the group
  int B = 1;
  std::mutex m;
  std::condition_variable cv;
  std::vector<Handle*> owner;       // slot -> attached handle (null: free)
  std::vector<char> ready;
  std::vector<const double*> vin;
  std::vector<double*> zout;
  std::vector<cudaStream_t> hs;
  std::vector<cudaEvent_t> ev_in;
  cudaEvent_t ev_done = nullptr;
  int active = 0, nready = 0;
  unsigned long long gen = 0;
  cudaError_t round_err = cudaSuccess;
  long long rounds = 0, slot_vcycles = 0, launches_batched = 0;
  int wait_us = 200;
  ~Group() {
    for (auto e : ev_in) if (e) cudaEventDestroy(e);
    if (ev_done) cudaEventDestroy(ev_done);
    if (core) stmg_destroy(reinterpret_cast<stmg_handle*>(core));
    if (stream) cudaStreamDestroy(stream);
  }
};

template <typename T>
static MG<T>& core_mg(Group& g);
template <>
MG<float>& core_mg<float>(Group& g) { return *g.core->mg32; }
template <>
MG<double>& core_mg<double>(Group& g) { return *g.core->mg64; }

// One batched V-cycle for every ready slot (caller holds the lock).
template <typename T>
static cudaError_t launch_round(Group& g) {
  MG<T>& mg = core_mg<T>(g);
  cudaStream_t gs = g.core->stream;
  const int64_t n0 = g.core->levels[0].Nst;
  int slots = 0;
  for (int j = 0; j < g.B; ++j) if (g.ready[j]) slots = j + 1;
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < slots && e == cudaSuccess; ++j) {
    if (!g.ready[j]) continue;
    e = cudaStreamWaitEvent(gs, g.ev_in[j], 0);
    if (e == cudaSuccess) e = vcopy<double, T>(n0, g.vin[j], mg.r[0] + j * n0, gs);
  }
  const long long l0 = launch_count();
  if (e == cudaSuccess) {
    bool done = false;
    if (mg.use_graph) {
      e = mg.vcycle_graph(slots);
      if (e == cudaSuccess) done = true;
      else { cudaGetLastError(); mg.use_graph = false; mg.drop_graph(); e = cudaSuccess; }
    }
    if (!done) e = mg.vcycle(mg.r[0], mg.z[0], slots);
  }
  g.launches_batched += launch_count() - l0;
  for (int j = 0; j < slots && e == cudaSuccess; ++j)
    if (g.ready[j]) e = vcopy<T, double>(n0, mg.z[0] + j * n0, g.zout[j], gs);
  if (e == cudaSuccess) e = cudaEventRecord(g.ev_done, gs);
  for (int j = 0; j < slots && e == cudaSuccess; ++j)
    if (g.ready[j]) e = cudaStreamWaitEvent(g.hs[j], g.ev_done, 0);
  ++g.rounds;
  g.slot_vcycles += g.nready;
  for (int j = 0; j < g.B; ++j) g.ready[j] = 0;
  g.nready = 0;
  g.round_err = e;
  ++g.gen;
  g.cv.notify_all();
  return e;
}

static cudaError_t launch_round_any(Group& g) {
  return g.core->precond_fp32() ? launch_round<float>(g) : launch_round<double>(g);
}

cudaError_t group_vcycle(Handle* h, const double* v, double* z) {
  Group& g = *h->group;
  std::unique_lock<std::mutex> lk(g.m);
  const int b = h->slot;
  cudaError_t e = cudaEventRecord(g.ev_in[b], h->stream);
  if (e != cudaSuccess) return e;
  g.vin[b] = v;
  g.zout[b] = z;
  g.hs[b] = h->stream;
  g.ready[b] = 1;
  ++g.nready;
  const unsigned long long my = g.gen;
  if (g.nready < g.active)
    g.cv.wait_for(lk, std::chrono::microseconds(g.wait_us), [&] { return g.gen != my; });
  if (g.gen == my) return launch_round_any(g);     // everyone in, or the others are late
  return g.round_err;
}

cudaError_t group_build(Handle* h, const double* U) {
  Group& g = *h->group;
  std::lock_guard<std::mutex> lk(g.m);
  cudaError_t e = cudaEventRecord(g.ev_in[h->slot], h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(g.core->stream, g.ev_in[h->slot], 0);
  if (e != cudaSuccess) return e;
  // runs on the group stream and ends with its synchronisation
  return g.core->precond_fp32() ? g.core->mg32->setup(U, h->slot, &h->pb) : g.core->mg64->setup(U, h->slot, &h->pb);
}

template <>
MG<float>* group_core_mg<float>(Handle* h) { return h->group->core->mg32.get(); }
template <>
MG<double>* group_core_mg<double>(Handle* h) { return h->group->core->mg64.get(); }

void group_forget(Handle* h) {
  if (!h->group) return;
  Group& g = *h->group;
  std::lock_guard<std::mutex> lk(g.m);
  g.owner[h->slot] = nullptr;
  h->group = nullptr;
  h->slot = -1;
}

void group_enter(Handle* h) {
  std::lock_guard<std::mutex> lk(h->group->m);
  ++h->group->active;
}

void group_leave(Handle* h) {
  Group& g = *h->group;
  std::lock_guard<std::mutex> lk(g.m);
  --g.active;
  // the remaining participants may all be waiting already
  if (g.nready > 0 && g.nready >= g.active) launch_round_any(g);
}

// Same shape: level sizes, orders, hierarchy and smoother options, slab length and mesh.
static bool compatible(const Handle* a, const Handle* b) {
  const stmg_params& p = a->prm;
  const stmg_params& q = b->prm;
  return p.dim == q.dim && p.n_cells_1d == q.n_cells_1d && p.r == q.r && p.k == q.k && p.n_levels_h == q.n_levels_h &&
         p.precond_precision == q.precond_precision && p.keep_time_degree == q.keep_time_degree &&
         p.smoother == q.smoother && p.vanka_fp16 == q.vanka_fp16 && p.nu1 == q.nu1 && p.nu2 == q.nu2 &&
         p.nu_tc == q.nu_tc && p.omega == q.omega && p.omega_p == q.omega_p && a->pb.tau == b->pb.tau &&
         p.gamma1 == q.gamma1 && p.gamma2 == q.gamma2 && p.bconv == q.bconv && a->verts0 == b->verts0;
}

}  // namespace stmg

using namespace stmg;

extern "C" {

stmg_status stmg_group_create(const stmg_params* p, const double* vertices, int slots, stmg_group** out) {
  if (!p || !out || slots < 1 || slots > 16) return STMG_ERR_ARG;
  *out = nullptr;
  auto g = std::make_unique<Group>();
  if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
    g->stream = nullptr;
    cudaGetLastError();
    return STMG_ERR_CUDA;
  }
  stmg_handle* hh = nullptr;
  stmg_status st = stmg_create(p, vertices, reinterpret_cast<stmg_stream>(g->stream), &hh);
  if (st != STMG_OK) return st;
  g->core = reinterpret_cast<Handle*>(hh);
  g->B = slots;
  cudaError_t e;
  if (g->core->precond_fp32()) {
    g->core->mg32.reset(new MG<float>());
    e = g->core->mg32->allocate(g->core, slots);
  } else {
    g->core->mg64.reset(new MG<double>());
    e = g->core->mg64->allocate(g->core, slots);
  }
  if (e == cudaErrorMemoryAllocation) return STMG_ERR_OOM;
  if (e != cudaSuccess) return STMG_ERR_CUDA;
  if (g->core->precond_fp32() ? !g->core->mg32->smoothable : !g->core->mg64->smoothable) return STMG_ERR_UNSUPPORTED;
  g->owner.assign(slots, nullptr);
  g->ready.assign(slots, 0);
  g->vin.assign(slots, nullptr);
  g->zout.assign(slots, nullptr);
  g->hs.assign(slots, nullptr);
  g->ev_in.assign(slots, nullptr);
  for (int j = 0; j < slots; ++j)
    if (cudaEventCreateWithFlags(&g->ev_in[j], cudaEventDisableTiming) != cudaSuccess) return STMG_ERR_CUDA;
  if (cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming) != cudaSuccess) return STMG_ERR_CUDA;
  *out = reinterpret_cast<stmg_group*>(g.release());
  return STMG_OK;
}

void stmg_group_destroy(stmg_group* gg) {
  Group* g = reinterpret_cast<Group*>(gg);
  if (!g) return;
  for (Handle* h : g->owner)
    if (h) { h->group = nullptr; h->slot = -1; }
  cudaStreamSynchronize(g->core->stream);
  delete g;
}

stmg_status stmg_group_attach(stmg_group* gg, stmg_handle* hh) {
  Group* g = reinterpret_cast<Group*>(gg);
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!g || !h) return STMG_ERR_ARG;
  if (h->group) return h->fail(STMG_ERR_ARG, "group_attach: the handle is attached to a group already");
  if (!compatible(g->core, h)) return h->fail(STMG_ERR_ARG, "group_attach: the handle's shape differs from the group's");
  std::lock_guard<std::mutex> lk(g->m);
  for (int j = 0; j < g->B; ++j)
    if (!g->owner[j]) {
      g->owner[j] = h;
      h->group = g;
      h->slot = j;
      return STMG_OK;
    }
  return h->fail(STMG_ERR_ARG, "group_attach: no free slot");
}

stmg_status stmg_group_detach(stmg_group* gg, stmg_handle* hh) {
  Group* g = reinterpret_cast<Group*>(gg);
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!g || !h || h->group != g) return STMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(g->m);
  g->owner[h->slot] = nullptr;
  h->group = nullptr;
  h->slot = -1;
  return STMG_OK;
}

stmg_status stmg_group_stats(const stmg_group* gg, long long* rounds, long long* slot_vcycles,
                             long long* launches) {
  const Group* g = reinterpret_cast<const Group*>(gg);
  if (!g) return STMG_ERR_ARG;
  if (rounds) *rounds = g->rounds;
  if (slot_vcycles) *slot_vcycles = g->slot_vcycles;
  if (launches) *launches = g->launches_batched;
  return STMG_OK;
}

}  // extern "C"
