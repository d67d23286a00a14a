// C ABI entry points: handle life cycle, hierarchy construction, operator apply, residual.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include <algorithm>
#include <array>
#include <atomic>

#include "../../include/stmg.h"
#include "counters.hpp"
#include "handle.hpp"
#include "userdata.hpp"
#include "group.hpp"

using namespace stmg;

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace stmg {

static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int height(int x) { int h = 0; while (x > 1) { x /= 2; ++h; } return h; }

// (r, k) of the p-levels, finest first (Sec. 4.2): the taller of the space and time degree
// hierarchies is halved alone until the heights match, then both, down to (1, 1); with
// keep_time the time degree stays k and only r is halved.
std::vector<std::pair<int, int>> p_hierarchy(int r, int k, int keep_time) {
  std::vector<std::pair<int, int>> pk{{r, k}};
  while (height(r) > 0 || (!keep_time && height(k) > 0)) {
    if (keep_time || height(r) > height(k)) r /= 2;
    else if (height(k) > height(r)) k /= 2;
    else { r /= 2; k /= 2; }
    pk.push_back({r, k});
  }
  return pk;
}

stmg_status Handle::fail(stmg_status s, const std::string& msg) {
  err = msg;
  return s;
}

void* Handle::dalloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); throw std::bad_alloc(); }
  allocs.push_back(p);
  return p;
}

void Handle::upload(void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) { cudaGetLastError(); throw CudaFailure(e); }
}

Handle::~Handle() {
  for (void* p : allocs) cudaFree(p);
}

static void build_level(Handle* h, Level& lv, const std::vector<double>& verts) {
  lv.N1 = (lv.r + 1) * lv.n + 1;
  lv.nnodes = 1;
  for (int l = 0; l < lv.d; ++l) lv.nnodes *= lv.N1;
  lv.tabs.build(lv.d, lv.r, lv.k);
  lv.npc = lv.tabs.npc;
  lv.Nv = lv.d * lv.nnodes;
  int64_t ncells = 1;
  for (int l = 0; l < lv.d; ++l) ncells *= lv.n;
  lv.Np = ncells * lv.npc;
  lv.Nst = (int64_t)(lv.k + 1) * (lv.Nv + lv.Np);
  lv.verts64 = (double*)h->dalloc(verts.size() * sizeof(double));
  lv.verts32 = (float*)h->dalloc(verts.size() * sizeof(float));
  std::vector<float> v32(verts.begin(), verts.end());
  h->upload(lv.verts64, verts.data(), verts.size() * sizeof(double));
  h->upload(lv.verts32, v32.data(), v32.size() * sizeof(float));
  lv.ncolors = 1 << lv.d;
  for (int c = 0; c < lv.ncolors; ++c) {
    ColorInfo& ci = lv.colors[c];
    ci.color = c;
    ci.count = 1;
    for (int l = 0; l < 3; ++l) ci.cnt[l] = 1;
    for (int l = 0; l < lv.d; ++l) {
      int bit = (c >> l) & 1;
      ci.cnt[l] = (lv.n - bit + 1) / 2;
      ci.count *= ci.cnt[l];
    }
    std::vector<int> bc;
    for (int64_t cell = 0; cell < ncells; ++cell) {
      int64_t rem = cell;
      bool bnd = false, match = true;
      for (int l = 0; l < lv.d; ++l) {
        int x = (int)(rem % lv.n); rem /= lv.n;
        if (x == 0 || x == lv.n - 1) bnd = true;
        if ((x & 1) != ((c >> l) & 1)) match = false;
      }
      if (bnd && match) bc.push_back((int)cell);
    }
    lv.nbcells[c] = (int)bc.size();
    lv.bcells[c] = (int*)h->dalloc(bc.size() * sizeof(int));
    h->upload(lv.bcells[c], bc.data(), bc.size() * sizeof(int));
  }
  if (lv.d == 2) {
    // geometry table of the 2D Jacobian apply (5 values per cell and Gauss point, both precisions)
    const size_t ng = (size_t)ncells * 5 * (lv.r + 2) * (lv.r + 2);
    lv.geo64 = (double*)h->dalloc(ng * sizeof(double));
    lv.geo32 = (float*)h->dalloc(ng * sizeof(float));
    if (build_geometry(lv, h->pb, h->stream) != cudaSuccess) throw CudaFailure(cudaErrorLaunchFailure);
  }
}

static std::vector<double> coarsen_vertices(const std::vector<double>& v, int d, int n) {
  int nc = n / 2;
  std::vector<double> out;
  int M = n + 1, Mc = nc + 1;
  int64_t tot = 1;
  for (int l = 0; l < d; ++l) tot *= Mc;
  out.resize(tot * d);
  for (int64_t i = 0; i < tot; ++i) {
    int64_t rem = i, src = 0, s = 1;
    for (int l = 0; l < d; ++l) { int x = (int)(rem % Mc); rem /= Mc; src += (int64_t)(2 * x) * s; s *= M; }
    for (int j = 0; j < d; ++j) out[i * d + j] = v[src * d + j];
  }
  return out;
}

}  // namespace stmg

extern "C" {

void stmg_params_default(stmg_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->dim = 2; p->n_cells_1d = 8; p->r = 1; p->k = 1;
  p->nu = 1e-2; p->tau = 0.1; p->gamma1 = 10.0; p->gamma2 = 10.0;
  p->problem = STMG_TG2D; p->bconv = 1; p->n_levels_h = -1;
  p->precond_precision = STMG_FP32;
  p->nu1 = 1; p->nu2 = 1; p->omega = 0.0;
  p->newton_rtol = 1e-8; p->newton_atol = 1e-12; p->newton_maxit = 20;
  p->ew_eta0 = 0.4; p->ew_c = 0.5; p->ew_theta = 1.5; p->ew_min = 1e-3; p->ew_max = 0.8;
  p->ls_lambda0 = 1.0; p->ls_c = 1e-4; p->ls_tau = 0.5; p->ls_alpha_min = 1e-3;
  p->ls_maxbt = 5; p->ls_window = 5;
  p->gmres_restart = 50; p->gmres_maxit = 50;
  p->rebuild_thetaN = 1.0; p->rebuild_thetaL = 2.0; p->rebuild_kappa_abs = 50;
  p->stag_s = 3; p->stag_theta = 0.95;
  p->omega_p = 1.0;
  p->vanka_fp16 = 0;
  p->build_chunk_cells = 0;
}

stmg_status stmg_footprint(const stmg_params* p, uint64_t* bytes) {
  if (!p || !bytes) return STMG_ERR_ARG;
  if (p->dim < 2 || p->dim > 3 || p->r < 1 || p->r > 3 || p->k < 0 || p->k > 2 || p->n_cells_1d < 1)
    return STMG_ERR_ARG;
  const int d = p->dim, n = p->n_cells_1d;
  std::vector<std::array<int, 3>> lv;     // (n, r, k) of every level, same rule as stmg_create
  for (auto& rk : p_hierarchy(p->r, p->k, p->keep_time_degree)) lv.push_back({n, rk.first, rk.second});
  const int r = lv.back()[1], k = lv.back()[2];
  int nn = n, hl = 0;
  while (nn % 2 == 0 && nn / 2 >= 2 && (p->n_levels_h < 0 || hl < p->n_levels_h)) { nn /= 2; ++hl; lv.push_back({nn, r, k}); }
  const double es = p->precond_precision == STMG_FP32 ? 4.0 : 8.0;
  double tot = 0, ea = 0, eb = 0, em = 0, nvmax = 0, wk = 0;
  std::vector<double> nst(lv.size());
  for (size_t l = 0; l < lv.size(); ++l) {
    const int ln = lv[l][0], lr = lv[l][1], lk = lv[l][2];
    double N1 = (lr + 1.0) * ln + 1.0, nodes = std::pow(N1, d), cells = std::pow((double)ln, d);
    double npc = (d == 2) ? (lr + 1.0) * (lr + 2.0) / 2.0 : (lr + 1.0) * (lr + 2.0) * (lr + 3.0) / 6.0;
    double Nv = d * nodes, Np = cells * npc;
    nst[l] = (lk + 1.0) * (Nv + Np);
    tot += 12.0 * std::pow(ln + 1.0, d) + 4.0 * cells;                  // vertices, boundary lists
    if (d == 2) tot += cells * 5.0 * (lr + 2.0) * (lr + 2.0) * 12.0;    // 2D geometry tables
    tot += 5.0 * nst[l] * es;                                            // level vectors
    if (l + 1 < lv.size()) {
      double nl = std::pow(lr + 2.0, d), mv = d * nl, msp = mv + npc;
      const int esz = p->vanka_fp16 ? 2 : (int)es;
      int sti = (int)msp;                                                // padded column stride
      while (((long long)msp * sti * esz) % 16 != 0) ++sti;
      const double ent = (lk + 1.0) * msp * sti;                         // time-diagonalised inverse
      if (p->smoother == 1)                                              // diagonal blobs
        tot += cells * es * (mv * (lk + 1.0) * (lk + 1.0) + npc * mv + (lk + 1.0) * npc * (lk + 1.0) * npc);
      else if (p->smoother == 2) {                                       // whole space-time inverse
        const double mst = (lk + 1.0) * msp;
        int stx = (int)mst;
        while (((long long)mst * stx * (int)es) % 16 != 0) ++stx;
        tot += cells * mst * stx * es;
      } else
        tot += p->vanka_fp16 ? cells * (ent * 2.0 + 4.0 * (lk + 1.0)) : cells * ent * es;  // patch inverses
      // element-matrix scratch: chunks of cell planes, at most ~2^18 cells and 8 GiB of FP64
      // element matrices (three planes at least)
      const double plane = cells / ln;
      double cap = p->build_chunk_cells > 0 ? (double)p->build_chunk_cells : 262144.0;
      cap = std::min(cap, std::floor(8.0 * 1073741824.0 / (8.0 * (mv * mv + npc * mv + nl * nl))));
      const double ec = cells <= cap ? cells : std::min(cells, std::max(3.0, std::floor(cap / plane)) * plane);
      ea = std::max(ea, ec * mv * mv * (p->smoother == 2 ? lk + 1.0 : 1.0));
      eb = std::max(eb, ec * npc * mv); em = std::max(em, ec * nl * nl);
      // patches beyond shared memory are factorised in a global workspace of 304 block slots
      const double pslot = 2.0 * msp * msp + mv * mv + nl * nl;
      if (p->smoother != 1 && es * (pslot + 2.0 * msp) + 4.0 * msp + 16.0 > 227.0 * 1024.0)
        wk = std::max(wk, 304.0 * pslot * es);
      // element tables beyond shared memory (3D Q4/P3) use 304 slots of the same workspace
      const double nf = std::pow(lr + 2.0, d - 1);
      const double etab = nl * nl * d + nl * nl + nl + nl * d + d * nl + d * (nf * (2.0 + 2.0 * d) + 2.0 * nf * nl) + 32.0;
      if (es * etab > 227.0 * 1024.0) wk = std::max(wk, 304.0 * etab * es);
      nvmax = std::max(nvmax, Nv);
      tot += 3.0 * std::max((lk + 1.0) * Nv, (lk + 1.0) * Np) * es;      // transfer scratch
    }
  }
  tot += (ea + eb + em + nvmax) * es + wk;
  const double Nc = nst.back(), Nb = Nc + lv.back()[2] + 1;
  tot += Nb * Nb * 16.0 + Nc * Nc * 8.0;                                 // coarse factors
  tot += (2.0 * p->gmres_restart + 1.0 + 9.0) * nst[0] * 8.0;           // Krylov basis, Newton vectors
  *bytes = (uint64_t)tot;
  return STMG_OK;
}

stmg_status stmg_set_physics(stmg_handle* hh, double nu, double tau, int problem) {
  if (!hh || !(nu > 0) || !(tau > 0) || problem < STMG_TG2D || problem > STMG_USER) return STMG_ERR_ARG;
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (h->group && tau != h->pb.tau) return h->fail(STMG_ERR_ARG, "set_physics: an attached handle keeps its group's tau");
  h->prm.nu = nu; h->prm.tau = tau; h->prm.problem = problem;
  h->pb.nu = nu; h->pb.tau = tau; h->pb.problem = problem;
  h->pb.ftab = problem == STMG_USER ? h->ftab : nullptr;
  h->pb.gtab = problem == STMG_USER ? h->gtab : nullptr;
  h->user_valid = false;                 // tau enters the Radau times of the data tables
  // the captured V-cycle bakes the physics into its kernel parameters
  if (h->mg32) h->mg32->drop_graph();
  if (h->mg64) h->mg64->drop_graph();
  return STMG_OK;
}

stmg_status stmg_create(const stmg_params* p, const double* vertices, stmg_stream stream,
                        stmg_handle** out) {
  if (!p || !out) return STMG_ERR_ARG;
  *out = nullptr;
  if (p->dim < 2 || p->dim > 3 || p->r < 1 || p->r > 3 || p->k < 0 || p->k > 2 ||
      p->n_cells_1d < 1 || p->n_cells_1d > 4096 || !(p->tau > 0) || !(p->nu > 0) ||
      p->problem < STMG_TG2D || p->problem > STMG_USER || p->smoother < 0 || p->smoother > 2)
    return STMG_ERR_ARG;
  auto h = std::make_unique<Handle>();
  h->prm = *p;
  // omega <= 0: 1.2 / 2^d -- each velocity vertex lies in up to 2^d of the additive patches
  if (!(h->prm.omega > 0)) h->prm.omega = 1.2 / (double)(1 << p->dim);
  h->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) { cudaGetLastError(); return STMG_ERR_CUDA; }
  h->pb = Problem{p->nu, p->tau, p->gamma1, p->gamma2, p->bconv, p->problem};
  const int d = p->dim, n = p->n_cells_1d;
  std::vector<double> verts;
  int64_t nv = 1;
  for (int l = 0; l < d; ++l) nv *= (n + 1);
  if (nv * d > ((int64_t)1 << 31)) return STMG_ERR_ARG;
  verts.resize(nv * d);
  if (vertices) {
    std::memcpy(verts.data(), vertices, verts.size() * sizeof(double));
  } else {
    for (int64_t i = 0; i < nv; ++i) {
      int64_t rem = i;
      for (int l = 0; l < d; ++l) { verts[i * d + l] = (double)(rem % (n + 1)) / n; rem /= (n + 1); }
    }
  }
  h->verts0 = verts;
  // hierarchy: p-coarsening first (taller of the r / k hierarchies alone until the heights
  // match, then both), then h-coarsening of the space mesh (Sec. 4.2, "cycle and coarsening order")
  try {
    std::vector<std::pair<int, int>> pk = p_hierarchy(p->r, p->k, p->keep_time_degree);
    const int r = pk.back().first, k = pk.back().second;
    const double p0 = p->r + 1;
    for (auto& rk : pk) {
      Level lv; lv.d = d; lv.n = n; lv.r = rk.first; lv.k = rk.second;
      lv.smoother = p->smoother;
      if (p->build_chunk_cells > 0) lv.chunk_cells = p->build_chunk_cells;
      lv.hscale = 1.0 / (p0 * (p0 + 1.0));
      build_level(h.get(), lv, verts);
      h->levels.push_back(lv);
    }
    int nn = n, hl = 0;
    std::vector<double> cv = verts;
    while (nn % 2 == 0 && nn / 2 >= 2 && (p->n_levels_h < 0 || hl < p->n_levels_h)) {
      cv = coarsen_vertices(cv, d, nn);
      nn /= 2; ++hl;
      Level lv; lv.d = d; lv.n = nn; lv.r = r; lv.k = k;
      lv.smoother = p->smoother;
      if (p->build_chunk_cells > 0) lv.chunk_cells = p->build_chunk_cells;
      lv.hscale = ((double)nn / n) / (p0 * (p0 + 1.0));
      build_level(h.get(), lv, cv);
      h->levels.push_back(lv);
    }
  } catch (const std::bad_alloc&) {
    return STMG_ERR_OOM;
  } catch (const CudaFailure&) {
    return STMG_ERR_CUDA;
  } catch (const std::exception&) {
    return STMG_ERR_ARG;
  }
  // only this handle's stream: a device-wide synchronisation would break graph captures that
  // other handles (serving workers) may have open on their streams
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) { cudaGetLastError(); return STMG_ERR_CUDA; }
  *out = reinterpret_cast<stmg_handle*>(h.release());
  return STMG_OK;
}

long long stmg_launch_count(void) { return launch_count(); }

stmg_status stmg_kernel_profile(const stmg_handle* hh, int cls, double* ms, long long* launches, double* bytes) {
  if (!hh || cls < 0 || cls >= KC_COUNT) return STMG_ERR_ARG;
  const Handle* h = reinterpret_cast<const Handle*>(hh);
  if (ms) *ms = h->kt[cls].ms;
  if (launches) *launches = h->kcount[cls];
  if (bytes) *bytes = h->kbytes[cls];
  return STMG_OK;
}

stmg_status stmg_kernel_profile_reset(stmg_handle* hh) {
  if (!hh) return STMG_ERR_ARG;
  Handle* h = reinterpret_cast<Handle*>(hh);
  for (int c = 0; c < KC_COUNT; ++c) { h->kt[c].ms = 0; h->kcount[c] = 0; h->kbytes[c] = 0; }
  return STMG_OK;
}

void stmg_destroy(stmg_handle* hh) {
  if (!hh) return;
  group_forget(reinterpret_cast<Handle*>(hh));
  delete reinterpret_cast<Handle*>(hh);
}

const char* stmg_last_error(const stmg_handle* hh) {
  if (!hh) return "null handle";
  return reinterpret_cast<const Handle*>(hh)->err.c_str();
}

stmg_status stmg_num_levels(const stmg_handle* hh, int* n_levels) {
  if (!hh || !n_levels) return STMG_ERR_ARG;
  *n_levels = (int)reinterpret_cast<const Handle*>(hh)->levels.size();
  return STMG_OK;
}

stmg_status stmg_level_info(const stmg_handle* hh, int level, int* n_cells_1d, int* r, int* k,
                            int64_t* n_v, int64_t* n_p, int64_t* n_st) {
  if (!hh) return STMG_ERR_ARG;
  const Handle* h = reinterpret_cast<const Handle*>(hh);
  if (level < 0 || level >= (int)h->levels.size()) return STMG_ERR_ARG;
  const Level& lv = h->levels[level];
  if (n_cells_1d) *n_cells_1d = lv.n;
  if (r) *r = lv.r;
  if (k) *k = lv.k;
  if (n_v) *n_v = lv.Nv;
  if (n_p) *n_p = lv.Np;
  if (n_st) *n_st = lv.Nst;
  return STMG_OK;
}

stmg_status stmg_apply(stmg_handle* hh, int level, int precision, const void* U_state,
                       const void* x, void* y) {
  if (!hh) return STMG_ERR_ARG;
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (level < 0 || level >= (int)h->levels.size() || !U_state || !x || !y || x == y || U_state == y)
    return h->fail(STMG_ERR_ARG, "stmg_apply: bad level or pointer");
  const Level& lv = h->levels[level];
  cudaError_t e;
  if (precision == STMG_FP64)
    e = launch_operator<double>(lv, h->pb, OP_JAC, 0.0, (const double*)x, (const double*)U_state,
                                nullptr, (double*)y, h->stream);
  else if (precision == STMG_FP32)
    e = launch_operator<float>(lv, h->pb, OP_JAC, 0.0, (const float*)x, (const float*)U_state,
                               nullptr, (float*)y, h->stream);
  else
    return h->fail(STMG_ERR_ARG, "stmg_apply: bad precision");
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("stmg_apply: ") + cudaGetErrorString(e));
  return STMG_OK;
}

stmg_status stmg_residual(stmg_handle* hh, double t_start, const double* U, const double* V_prev,
                          double* R) {
  if (!hh) return STMG_ERR_ARG;
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!U || !V_prev || !R || R == U) return h->fail(STMG_ERR_ARG, "stmg_residual: bad pointer");
  if (h->pb.problem == STMG_USER && !h->ftab)
    return h->fail(STMG_ERR_ARG, "stmg_residual: problem STMG_USER needs stmg_set_data first");
  cudaError_t e = refresh_user_data(h, t_start);
  if (e == cudaErrorInvalidValue) return h->fail(STMG_ERR_NUMERIC, "stmg_residual: a data callback returned a non-finite value");
  if (e == cudaSuccess) e = launch_operator<double>(h->levels[0], h->pb, OP_RES, t_start, U, nullptr, V_prev, R, h->stream);
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("stmg_residual: ") + cudaGetErrorString(e));
  return STMG_OK;
}

stmg_status stmg_initial_condition(stmg_handle* hh, stmg_field_fn v0, void* user, double* V0) {
  if (!hh) return STMG_ERR_ARG;
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!V0) return h->fail(STMG_ERR_ARG, "stmg_initial_condition: null pointer");
  if (v0) {
    // the caller's v0 at the velocity nodes of the finest level (GLL nodes of the mapped cells)
    const Level& L = h->levels[0];
    const int d = L.d, n = L.n, r1 = L.r + 1;
    const int64_t nn = L.nnodes;
    std::vector<double> xs((size_t)d * nn), out((size_t)d * nn, 0.0);
    for (int64_t gi = 0; gi < nn; ++gi) {
      int64_t rem = gi;
      int cc[3] = {0, 0, 0};
      double xh[3] = {0, 0, 0};
      for (int l = 0; l < d; ++l) {
        const int gm = (int)(rem % L.N1); rem /= L.N1;
        cc[l] = std::min(gm / r1, n - 1);
        xh[l] = L.tabs.gll[gm - cc[l] * r1];
      }
      double x[3] = {0, 0, 0};
      for (int c = 0; c < (1 << d); ++c) {
        double wgt = 1.0;
        int64_t v = 0, s = 1;
        for (int l = 0; l < d; ++l) {
          const int b = (c >> l) & 1;
          wgt *= b ? xh[l] : 1.0 - xh[l];
          v += (int64_t)(cc[l] + b) * s;
          s *= (n + 1);
        }
        for (int i = 0; i < d; ++i) x[i] += h->verts0[v * d + i] * wgt;
      }
      for (int i = 0; i < d; ++i) xs[(size_t)i * nn + gi] = x[i];
    }
    v0(user, nn, xs.data(), 0.0, out.data());
    for (double v : out)
      if (!std::isfinite(v)) return h->fail(STMG_ERR_NUMERIC, "stmg_initial_condition: v0 returned a non-finite value");
    try {
      h->upload(V0, out.data(), out.size() * sizeof(double));
    } catch (const CudaFailure& f) {
      return h->fail(STMG_ERR_CUDA, std::string("stmg_initial_condition: ") + cudaGetErrorString(f.err));
    }
    return STMG_OK;
  }
  if (h->pb.problem == STMG_USER) {
    cudaError_t e = cudaMemsetAsync(V0, 0, h->levels[0].Nv * sizeof(double), h->stream);
    if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("stmg_initial_condition: ") + cudaGetErrorString(e));
    return STMG_OK;
  }
  cudaError_t e = launch_initial_condition(h->levels[0], h->pb, V0, h->stream);
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("stmg_initial_condition: ") + cudaGetErrorString(e));
  return STMG_OK;
}

}  // extern "C"
