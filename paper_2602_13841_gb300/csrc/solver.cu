// Newton-FGMRES slab solver (Sec. 4.1, Alg. 1-2) with the hp-STMG preconditioner, and the
// C-ABI entry points of the smoother, V-cycle, transfers and slab solve.
//
// FGMRES (Saad 1993): right-preconditioned, flexible (one V-cycle per iteration), restart m,
// iteration cap; Arnoldi orthogonalisation by CGS2 (classical Gram-Schmidt with one full
// re-orthogonalisation, Giraud et al. 2005) on the device, Givens rotations in FP64 on the
// host (one device->host transfer of the Hessenberg column per iteration).  Stop when the
// Euclidean residual estimate |g_{j+1}| <= eta ||b||.
// Newton (Alg. 1): Eisenstat-Walker forcing, rebuild triggers, mass-weighted norm; Armijo
// (Alg. 2) with g0 = r^T M J dX, nonmonotone window of the last M merits of the slab,
// safeguarded quadratic / cubic interpolation, alpha_min accepted when nothing else is.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "handle.hpp"
#include "userdata.hpp"
#include "group.hpp"
#include "vec.cuh"
#include "counters.hpp"

namespace stmg {

#define CKE(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return e_; } while (0)

// ---------------------------------------------------------------------------- timers
cudaEvent_t PhaseTimer::get() {
  if (used == pool.size()) { cudaEvent_t e; cudaEventCreate(&e); pool.push_back(e); }
  return pool[used++];
}
void PhaseTimer::begin(cudaStream_t s) { open_ = get(); cudaEventRecord(open_, s); }
void PhaseTimer::end(cudaStream_t s) { cudaEvent_t e = get(); cudaEventRecord(e, s); spans.push_back({open_, e}); }
void PhaseTimer::collect() {
  for (auto& p : spans) { float m = 0; if (cudaEventElapsedTime(&m, p.first, p.second) == cudaSuccess) ms += m; }
  spans.clear();
  used = 0;
}
PhaseTimer::~PhaseTimer() { for (auto e : pool) cudaEventDestroy(e); }

// ---------------------------------------------------------------------------- set-up
cudaError_t Handle::ensure_mg() {
  if (group) return cudaSuccess;                 // the group's hierarchy serves this handle
  if (precond_fp32()) {
    if (!mg32) { mg32.reset(new MG<float>()); cudaError_t e = mg32->allocate(this); if (e != cudaSuccess) { mg32.reset(); return e; } }
  } else {
    if (!mg64) { mg64.reset(new MG<double>()); cudaError_t e = mg64->allocate(this); if (e != cudaSuccess) { mg64.reset(); return e; } }
  }
  return cudaSuccess;
}

__global__ void k_const_p0(double* e, int64_t poff, int64_t Np, int npc) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Np; i += (int64_t)gridDim.x * blockDim.x)
    e[poff + i] = (i % npc == 0) ? 1.0 : 0.0;
}

cudaError_t Handle::ensure_solver() {
  CKE(ensure_mg());
  if (solver_ready) return cudaSuccess;
  const Level& L = levels[0];
  const int m = prm.gmres_restart;
  if (m < 1 || m > 60) return cudaErrorInvalidValue;
  try {
    Vb = (double*)dalloc((size_t)(m + 1) * L.Nst * sizeof(double));
    Zb = (double*)dalloc((size_t)m * L.Nst * sizeof(double));
    w = (double*)dalloc(L.Nst * sizeof(double));
    R = (double*)dalloc(L.Nst * sizeof(double));
    dX = (double*)dalloc(L.Nst * sizeof(double));
    Xt = (double*)dalloc(L.Nst * sizeof(double));
    Mv = (double*)dalloc(L.Nst * sizeof(double));
    Jv = (double*)dalloc(L.Nst * sizeof(double));
    pw = (double*)dalloc(L.Nst * sizeof(double));
    scratch = (double*)dalloc((size_t)RED_BLOCKS * 64 * sizeof(double));
    hdev = (double*)dalloc(256 * sizeof(double));
    flag = (int*)dalloc(sizeof(int));
  } catch (const std::bad_alloc&) {
    return cudaErrorMemoryAllocation;
  }
  // pressure weights: pw = M e with e = constant pressure at time node 0 (its pressure part at
  // time node 0 holds w_0 * int psi_m over each cell)
  CKE(cudaMemsetAsync(Mv, 0, L.Nst * sizeof(double), stream));
  k_const_p0<<<64, 256, 0, stream>>>(Mv, (int64_t)(L.k + 1) * L.Nv, L.Np, L.npc);
  note_launch();
  CKE(launch_operator<double>(L, pb, OP_MASS, 0.0, Mv, nullptr, nullptr, pw, stream));
  solver_ready = true;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------- helpers
static cudaError_t dot_host(Handle* h, int64_t n, const double* a, const double* b, double* out) {
  CKE(vdots<double>(n, 1, a, n, b, h->hdev + 192, h->scratch, h->stream));
  CKE(cudaMemcpyAsync(out, h->hdev + 192, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return cudaStreamSynchronize(h->stream);
}

// ||Z||_M = sqrt(Z^T M Z)
static cudaError_t mnorm(Handle* h, const double* Z, double* out) {
  const Level& L = h->levels[0];
  h->kbegin(KC_MASS);
  CKE(launch_operator<double>(L, h->pb, OP_MASS, 0.0, Z, nullptr, nullptr, h->Mv, h->stream));
  h->kend(KC_MASS, 16.0 * L.Nst);
  double v = 0;
  CKE(dot_host(h, L.Nst, Z, h->Mv, &v));
  *out = std::sqrt(v > 0 ? v : 0.0);
  return cudaSuccess;
}

__global__ void k_sub_mean(double* P, int64_t Np, int npc, int kp1, const double* dots, double inv_vol) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (Np / npc) * kp1;
       i += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(i / (Np / npc));
    int64_t c = i % (Np / npc);
    P[a * Np + c * npc] -= dots[a] * inv_vol;
  }
}

// remove the pressure mean at every time node (L^2_0 representative)
static cudaError_t project_mean(Handle* h, double* U) {
  const Level& L = h->levels[0];
  const double* pwp = h->pw + (int64_t)(L.k + 1) * L.Nv;
  double* P = U + (int64_t)(L.k + 1) * L.Nv;
  CKE(vdots<double>(L.Np, L.k + 1, P, L.Np, pwp, h->hdev + 224, h->scratch, h->stream));
  // volume (times w_0): the dot of pw with the constant pressure (mode 0 = 1)
  double vol = 0;
  {
    CKE(cudaMemsetAsync(h->Mv, 0, L.Np * sizeof(double), h->stream));
    k_const_p0<<<64, 256, 0, h->stream>>>(h->Mv, 0, L.Np, L.npc);
  note_launch();
    CKE(dot_host(h, L.Np, pwp, h->Mv, &vol));
  }
  k_sub_mean<<<64, 256, 0, h->stream>>>(P, L.Np, L.npc, L.k + 1, h->hdev + 224, 1.0 / vol);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t precondition(Handle* h, MG<T>& mg, const double* v, double* z) {
  if (h->group) return group_vcycle(h, v, z);
  const Level& L = h->levels[0];
  CKE((vcopy<double, T>(L.Nst, v, mg.r[0], h->stream)));
  if (h->timing) h->t_mg.begin(h->stream);
  bool done = false;
  if (mg.use_graph && h->stream != nullptr) {
    cudaError_t e = mg.vcycle_graph();
    if (e == cudaSuccess) done = true;
    else { cudaGetLastError(); mg.use_graph = false; mg.drop_graph(); }   // fall back to direct launches
  }
  if (!done) CKE(mg.vcycle(mg.r[0], mg.z[0]));
  if (h->timing) h->t_mg.end(h->stream);
  CKE((vcopy<T, double>(L.Nst, mg.z[0], z, h->stream)));
  return cudaSuccess;
}

// FGMRES: solve J(U) x = b, x starts at 0.  its: iterations; ratios: |g_{j+1}| / |g_j|.
template <typename T>
static cudaError_t fgmres(Handle* h, MG<T>& mg, const double* U, const double* b, double* x, double tol,
                          int* its_out, std::vector<double>* ratios) {
  const Level& L = h->levels[0];
  const int64_t N = L.Nst;
  const int m = h->prm.gmres_restart, maxit = h->prm.gmres_maxit;
  cudaStream_t s = h->stream;
  CKE(cudaMemsetAsync(x, 0, N * sizeof(double), s));
  double bnorm2 = 0;
  CKE(dot_host(h, N, b, b, &bnorm2));
  const double bnorm = std::sqrt(bnorm2);
  int its = 0;
  if (bnorm == 0.0) { *its_out = 0; return cudaSuccess; }
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), hh(3 * 64);
  bool done = false;
  while (its < maxit && !done) {
    double beta;
    if (its == 0) {
      beta = bnorm;
      CKE(vscale<double>(N, 1.0 / beta, b, h->Vb, s));
    } else {
      CKE(launch_operator<double>(L, h->pb, OP_JAC, 0.0, x, U, nullptr, h->w, s));
      CKE(vaxpby<double>(N, 1.0, b, -1.0, h->w, s));
      double r2 = 0;
      CKE(dot_host(h, N, h->w, h->w, &r2));
      beta = std::sqrt(r2);
      if (beta <= tol * bnorm) break;
      CKE(vscale<double>(N, 1.0 / beta, h->w, h->Vb, s));
    }
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jd = 0;
    for (int j = 0; j < m && its < maxit; ++j) {
      double* vj = h->Vb + (int64_t)j * N;
      double* zj = h->Zb + (int64_t)j * N;
      CKE(precondition<T>(h, mg, vj, zj));
      // algorithmic bytes of the apply: read x and the state velocity, write y (FP64)
      h->kbegin(KC_APPLY64);
      CKE(launch_operator<double>(L, h->pb, OP_JAC, 0.0, zj, U, nullptr, h->w, s));
      h->kend(KC_APPLY64, 8.0 * (L.k + 1) * (3.0 * L.Nv + 2.0 * L.Np));
      // CGS2
      CKE(vdots<double>(N, j + 1, h->Vb, N, h->w, h->hdev, h->scratch, s));
      CKE(vsub_comb<double>(N, j + 1, h->Vb, N, h->hdev, h->w, s));
      CKE(vdots<double>(N, j + 1, h->Vb, N, h->w, h->hdev + 64, h->scratch, s));
      CKE(vsub_comb<double>(N, j + 1, h->Vb, N, h->hdev + 64, h->w, s));
      CKE(vdots<double>(N, 1, h->w, N, h->w, h->hdev + 128, h->scratch, s));
      CKE(cudaMemcpyAsync(hh.data(), h->hdev, 3 * 64 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CKE(cudaStreamSynchronize(s));
      if (h->timing && mg.graph_exec) mg.collect_graph_timers();
      for (int i = 0; i <= j; ++i) H[i * m + j] = hh[i] + hh[64 + i];
      const double hn = std::sqrt(hh[128] > 0 ? hh[128] : 0.0);
      H[(j + 1) * m + j] = hn;
      if (hn > 0) CKE(vscale<double>(N, 1.0 / hn, h->w, h->Vb + (int64_t)(j + 1) * N, s));
      for (int i = 0; i < j; ++i) {
        double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
        H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
        H[i * m + j] = t;
      }
      double den = std::hypot(H[j * m + j], H[(j + 1) * m + j]);
      cs[j] = den > 0 ? H[j * m + j] / den : 1.0;
      sn[j] = den > 0 ? H[(j + 1) * m + j] / den : 0.0;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      const double prev = std::fabs(g[j]);
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++its;
      jd = j + 1;
      if (ratios) ratios->push_back(std::fabs(g[j + 1]) / (prev > 1e-300 ? prev : 1e-300));
      if (!std::isfinite(g[j + 1])) return cudaErrorIllegalState;
      if (std::fabs(g[j + 1]) <= tol * bnorm) { done = true; break; }
      if (hn == 0.0) { done = true; break; }
    }
    std::vector<double> y(jd);
    for (int i = jd - 1; i >= 0; --i) {
      double acc = g[i];
      for (int k = i + 1; k < jd; ++k) acc -= H[i * m + k] * y[k];
      y[i] = acc / H[i * m + i];
    }
    CKE(vadd_comb_host(N, jd, h->Zb, N, y.data(), x, s));
  }
  *its_out = its;
  return cudaSuccess;
}

static double interp_step(double a1, double f1, bool have2, double a2, double f2, double phi0, double g0,
                          bool* ok) {
  *ok = true;
  if (!have2) {
    double den = 2.0 * (f1 - phi0 - g0 * a1);
    if (den <= 0) { *ok = false; return 0; }
    return -g0 * a1 * a1 / den;
  }
  double r1 = f1 - phi0 - g0 * a1, r2 = f2 - phi0 - g0 * a2, dd = a1 - a2;
  double a = (r1 / (a1 * a1) - r2 / (a2 * a2)) / dd;
  double b = (-a2 * r1 / (a1 * a1) + a1 * r2 / (a2 * a2)) / dd;
  if (a == 0.0) {
    if (b == 0.0) { *ok = false; return 0; }
    return -g0 / (2.0 * b);
  }
  double disc = b * b - 3.0 * a * g0;
  if (disc < 0) { *ok = false; return 0; }
  return (-b + std::sqrt(disc)) / (3.0 * a);
}

template <typename T>
static cudaError_t rebuild(Handle* h, MG<T>& mg, const double* X, stmg_stats* st) {
  if (h->timing) h->t_rebuild.begin(h->stream);
  cudaError_t e = h->group ? group_build(h, X) : mg.setup(X);
  if (h->timing) h->t_rebuild.end(h->stream);
  st->rebuilds++;
  return e;
}

template <typename T>
static stmg_status newton(Handle* h, MG<T>& mg, double t0, const double* Vprev, double* X, stmg_stats* st) {
  const Level& L = h->levels[0];
  const int64_t N = L.Nst;
  cudaStream_t s = h->stream;
  const stmg_params& P = h->prm;
  const double eps = 1e-30;
#define CKS(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return h->fail(e_ == cudaErrorUnknown ? STMG_ERR_NUMERIC : e_ == cudaErrorNotSupported ? STMG_ERR_UNSUPPORTED : STMG_ERR_CUDA, std::string("slab_solve: ") + #x + ": " + cudaGetErrorString(e_)); } while (0)
  {
    cudaError_t eu = refresh_user_data(h, t0);
    if (eu == cudaErrorInvalidValue) return h->fail(STMG_ERR_NUMERIC, "slab_solve: a data callback returned a non-finite value");
    CKS(eu);
  }
  CKS(launch_operator<double>(L, h->pb, OP_RES, t0, X, nullptr, Vprev, h->R, s));
  double nr = 0;
  CKS(mnorm(h, h->R, &nr));
  const double n0 = nr;
  st->res0 = n0;
  if (!std::isfinite(n0)) return h->fail(STMG_ERR_NUMERIC, "slab_solve: non-finite initial residual");
  double nprev = n0, eta = P.ew_eta0, rho_prev = 1.0;
  int kap_prev = 1, kap_ref = 1;
  std::vector<double> window{0.5 * n0 * n0};
  std::vector<double> hist{n0};                   // ||R||_M after every step (stall check)
  bool stalled = false;
  int k = 0;
  while (nr > std::max(P.newton_atol, P.newton_rtol * n0) && k < P.newton_maxit && !stalled) {
    if (rho_prev >= P.rebuild_thetaN || kap_prev >= std::max(P.rebuild_thetaL * kap_ref, (double)P.rebuild_kappa_abs)) {
      CKS(rebuild<T>(h, mg, X, st));
      kap_ref = std::max(1, kap_prev);
    }
    if (k > 0)
      eta = std::min(std::max(P.ew_c * eta * std::pow(nr / std::max(nprev, eps), P.ew_theta), P.ew_min), P.ew_max);
    // FGMRES on J dX = -R
    CKS(vscale<double>(N, -1.0, h->R, h->Jv, s));
    int kap = 0;
    std::vector<double> ratios;
    CKS(fgmres<T>(h, mg, X, h->Jv, h->dX, eta, &kap, &ratios));
    st->gmres_its_total += kap;
    // Armijo (Alg. 2): phi(alpha) = 1/2 ||R(X + alpha dX)||_M^2, g0 = R^T M J dX
    const double phi0 = 0.5 * nr * nr;
    CKS(launch_operator<double>(L, h->pb, OP_JAC, 0.0, h->dX, X, nullptr, h->Jv, s));
    CKS(launch_operator<double>(L, h->pb, OP_MASS, 0.0, h->Jv, nullptr, nullptr, h->Mv, s));
    double g0 = 0;
    CKS(dot_host(h, N, h->R, h->Mv, &g0));
    double alpha = P.ls_lambda0, phit = 0;
    bool accepted = false, have1 = false, have2 = false;
    double a1 = 0, f1 = 0, a2 = 0, f2 = 0;
    for (int bt = 0; bt <= P.ls_maxbt; ++bt) {
      if (alpha <= P.ls_alpha_min) break;
      CKS(cudaMemcpyAsync(h->Xt, X, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CKS(vaxpby<double>(N, alpha, h->dX, 1.0, h->Xt, s));
      CKS(launch_operator<double>(L, h->pb, OP_RES, t0, h->Xt, nullptr, Vprev, h->w, s));
      double nt = 0;
      CKS(mnorm(h, h->w, &nt));
      phit = 0.5 * nt * nt;
      double phimax = phi0;
      if (P.ls_window > 0) for (double v : window) phimax = std::max(phimax, v);
      if (std::isfinite(phit) && phit <= phimax + P.ls_c * alpha * g0) { accepted = true; break; }
      if (have1) { a2 = a1; f2 = f1; have2 = true; }
      a1 = alpha; f1 = std::isfinite(phit) ? phit : 1e300; have1 = true;
      st->armijo_backtracks++;
      bool ok = false;
      double ai = interp_step(a1, f1, have2, a2, f2, phi0, g0, &ok);
      alpha = (!ok || !std::isfinite(ai)) ? alpha * P.ls_tau : std::min(std::max(ai, 0.1 * alpha), 0.5 * alpha);
    }
    if (!accepted) {
      alpha = std::max(alpha, P.ls_alpha_min);
      CKS(cudaMemcpyAsync(h->Xt, X, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CKS(vaxpby<double>(N, alpha, h->dX, 1.0, h->Xt, s));
      CKS(launch_operator<double>(L, h->pb, OP_RES, t0, h->Xt, nullptr, Vprev, h->w, s));
      double nt = 0;
      CKS(mnorm(h, h->w, &nt));
      phit = 0.5 * nt * nt;
    }
    window.push_back(phit);
    const size_t W = (size_t)std::max(P.ls_window, 1);
    if (window.size() > W) window.erase(window.begin(), window.end() - W);
    CKS(vaxpby<double>(N, alpha, h->dX, 1.0, X, s));
    CKS(project_mean(h, X));
    nprev = nr;
    CKS(launch_operator<double>(L, h->pb, OP_RES, t0, X, nullptr, Vprev, h->R, s));
    CKS(mnorm(h, h->R, &nr));
    if (!std::isfinite(nr)) return h->fail(STMG_ERR_NUMERIC, "slab_solve: non-finite residual");
    rho_prev = nr / std::max(nprev, eps);
    kap_prev = std::max(1, kap);
    const int sw = P.stag_s;
    if (sw > 0 && (int)ratios.size() >= sw) {
      bool stag = true;
      for (int i = (int)ratios.size() - sw; i < (int)ratios.size(); ++i) stag = stag && ratios[i] >= P.stag_theta;
      if (stag) CKS(rebuild<T>(h, mg, X, st));
    }
    ++k;
    hist.push_back(nr);
    const int ss = P.newton_stall_steps;
    if (ss > 0 && (int)hist.size() > ss && nr > P.newton_stall_ratio * hist[hist.size() - 1 - ss]) stalled = true;
  }
  st->newton_its = k;
  st->res_final = nr;
#undef CKS
  if (nr > std::max(P.newton_atol, P.newton_rtol * n0))
    return h->fail(STMG_ERR_NOT_CONVERGED, stalled ? "slab_solve: Newton stalled (no progress over newton_stall_steps steps)"
                                                   : "slab_solve: Newton reached its iteration cap");
  return STMG_OK;
}

}  // namespace stmg

using namespace stmg;

static Handle* H(stmg_handle* hh) { return reinterpret_cast<Handle*>(hh); }

extern "C" {

stmg_status stmg_smoother_build(stmg_handle* hh, const double* U) {
  if (!hh || !U) return STMG_ERR_ARG;
  Handle* h = H(hh);
  cudaError_t e = h->ensure_mg();
  if (e == cudaErrorNotSupported) return h->fail(STMG_ERR_UNSUPPORTED, "smoother_build: patch too large for this configuration");
  if (e != cudaSuccess) return h->fail(e == cudaErrorMemoryAllocation ? STMG_ERR_OOM : STMG_ERR_CUDA, std::string("smoother_build: ") + cudaGetErrorString(e));
  e = h->group ? group_build(h, U) : h->precond_fp32() ? h->mg32->setup(U) : h->mg64->setup(U);
  if (e == cudaErrorUnknown) return h->fail(STMG_ERR_NUMERIC, "smoother_build: singular patch or coarse matrix");
  if (e == cudaErrorNotSupported) return h->fail(STMG_ERR_UNSUPPORTED, "smoother_build: patch too large for this configuration");
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("smoother_build: ") + cudaGetErrorString(e));
  return STMG_OK;
}

stmg_status stmg_smoother_sweep(stmg_handle* hh, int level, const void* rhs, void* d, int nsweeps, int zero_start) {
  if (!hh || !rhs || !d || nsweeps < 0) return STMG_ERR_ARG;
  Handle* h = H(hh);
  if (h->group) return h->fail(STMG_ERR_ARG, "smoother_sweep: the handle is attached to a group");
  if (level < 0 || level + 1 >= (int)h->levels.size()) return h->fail(STMG_ERR_ARG, "smoother_sweep: level has no smoother");
  bool built = h->precond_fp32() ? (h->mg32 && h->mg32->built) : (h->mg64 && h->mg64->built);
  if (!built) return h->fail(STMG_ERR_ARG, "smoother_sweep: call stmg_smoother_build first");
  cudaError_t e = h->precond_fp32() ? h->mg32->sweep(level, (const float*)rhs, (float*)d, nsweeps, zero_start != 0)
                                    : h->mg64->sweep(level, (const double*)rhs, (double*)d, nsweeps, zero_start != 0);
  if (e == cudaSuccess) e = h->precond_fp32() ? h->mg32->check_wait() : h->mg64->check_wait();
  if (e == cudaErrorTimeout) return h->fail(STMG_ERR_TIMEOUT, "smoother_sweep: a bounded wait in the Vanka apply ran out");
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("smoother_sweep: ") + cudaGetErrorString(e));
  return STMG_OK;
}

stmg_status stmg_vcycle(stmg_handle* hh, const double* r, double* z) {
  if (!hh || !r || !z) return STMG_ERR_ARG;
  Handle* h = H(hh);
  if (h->group) return h->fail(STMG_ERR_ARG, "vcycle: the handle is attached to a group");
  bool built = h->precond_fp32() ? (h->mg32 && h->mg32->built) : (h->mg64 && h->mg64->built);
  if (!built) return h->fail(STMG_ERR_ARG, "vcycle: call stmg_smoother_build first");
  cudaError_t e = h->precond_fp32() ? precondition<float>(h, *h->mg32, r, z) : precondition<double>(h, *h->mg64, r, z);
  if (e == cudaSuccess) e = h->precond_fp32() ? h->mg32->check_wait() : h->mg64->check_wait();
  if (e == cudaErrorTimeout) return h->fail(STMG_ERR_TIMEOUT, "vcycle: a bounded wait in the Vanka apply ran out");
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("vcycle: ") + cudaGetErrorString(e));
  return STMG_OK;
}

stmg_status stmg_transfer(stmg_handle* hh, int level, int op, const void* in, void* out) {
  if (!hh || !in || !out) return STMG_ERR_ARG;
  Handle* h = H(hh);
  if (h->group) return h->fail(STMG_ERR_ARG, "transfer: the handle is attached to a group");
  if (level < 0 || level + 1 >= (int)h->levels.size() || op < 0 || op > 2) return h->fail(STMG_ERR_ARG, "transfer: bad level or op");
  cudaError_t e = h->ensure_mg();
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("transfer: ") + cudaGetErrorString(e));
  if (h->precond_fp32()) {
    const Transfer& t = h->mg32->tr[level];
    e = op == 0 ? t.prolong<float>((const float*)in, (float*)out, h->stream)
      : op == 1 ? t.restrict_<float>((const float*)in, (float*)out, h->stream)
                : t.interp_state<float>((const float*)in, (float*)out, h->stream);
  } else {
    const Transfer& t = h->mg64->tr[level];
    e = op == 0 ? t.prolong<double>((const double*)in, (double*)out, h->stream)
      : op == 1 ? t.restrict_<double>((const double*)in, (double*)out, h->stream)
                : t.interp_state<double>((const double*)in, (double*)out, h->stream);
  }
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("transfer: ") + cudaGetErrorString(e));
  return STMG_OK;
}

stmg_status stmg_level_state(stmg_handle* hh, int level, void* out) {
  if (!hh || !out) return STMG_ERR_ARG;
  Handle* h = H(hh);
  if (h->group) return h->fail(STMG_ERR_ARG, "level_state: the handle is attached to a group");
  if (level < 0 || level >= (int)h->levels.size()) return h->fail(STMG_ERR_ARG, "level_state: bad level");
  bool built = h->precond_fp32() ? (h->mg32 && h->mg32->built) : (h->mg64 && h->mg64->built);
  if (!built) return h->fail(STMG_ERR_ARG, "level_state: call stmg_smoother_build first");
  const Level& lv = h->levels[level];
  size_t es = h->precond_fp32() ? sizeof(float) : sizeof(double);
  const void* src = h->precond_fp32() ? (const void*)h->mg32->U[level] : (const void*)h->mg64->U[level];
  cudaError_t e = cudaMemcpyAsync(out, src, lv.Nst * es, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, "level_state: copy failed");
  return STMG_OK;
}

stmg_status stmg_mass(stmg_handle* hh, const double* x, double* y) {
  if (!hh || !x || !y || x == y) return STMG_ERR_ARG;
  Handle* h = H(hh);
  cudaError_t e = launch_operator<double>(h->levels[0], h->pb, OP_MASS, 0.0, x, nullptr, nullptr, y, h->stream);
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("mass: ") + cudaGetErrorString(e));
  return STMG_OK;
}

__global__ void k_guess(const double* Vp, double* U, int64_t Nv, int kp1, int64_t Nst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nst; i += (int64_t)gridDim.x * blockDim.x)
    U[i] = (i < kp1 * Nv) ? Vp[i % Nv] : 0.0;
}

stmg_status stmg_initial_guess(stmg_handle* hh, const double* V_prev, double* U) {
  if (!hh || !V_prev || !U) return STMG_ERR_ARG;
  Handle* h = H(hh);
  const Level& L = h->levels[0];
  k_guess<<<152 * 8, 256, 0, h->stream>>>(V_prev, U, L.Nv, L.k + 1, L.Nst);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return h->fail(STMG_ERR_CUDA, std::string("initial_guess: ") + cudaGetErrorString(e));
  return STMG_OK;
}

stmg_status stmg_set_timing(stmg_handle* hh, int on) {
  if (!hh) return STMG_ERR_ARG;
  H(hh)->timing = on != 0;
  return STMG_OK;
}

stmg_status stmg_test_wait_timeout(stmg_handle* hh, int on) {
  if (!hh) return STMG_ERR_ARG;
  Handle* h = H(hh);
  h->wait_fault = on != 0;
  // captured V-cycles bake the kernel arguments in
  if (h->mg32) h->mg32->drop_graph();
  if (h->mg64) h->mg64->drop_graph();
  return STMG_OK;
}

stmg_status stmg_set_timing_classes(stmg_handle* hh, unsigned mask) {
  if (!hh) return STMG_ERR_ARG;
  H(hh)->kmask = mask;
  return STMG_OK;
}

stmg_status stmg_slab_solve(stmg_handle* hh, double t_start, const double* V_prev, double* U, stmg_stats* st) {
  if (!hh || !V_prev || !U) return STMG_ERR_ARG;
  Handle* h = H(hh);
  stmg_stats local{};
  stmg_stats* S = st ? st : &local;
  std::memset(S, 0, sizeof(*S));
  cudaError_t e = h->ensure_solver();
  if (e == cudaErrorNotSupported) return h->fail(STMG_ERR_UNSUPPORTED, "slab_solve: patch too large for this configuration");
  if (e != cudaSuccess) return h->fail(e == cudaErrorMemoryAllocation ? STMG_ERR_OOM : STMG_ERR_CUDA, std::string("slab_solve: ") + cudaGetErrorString(e));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double vanka0 = 0;
  if (h->timing) {
    for (int c = 0; c < KC_COUNT; ++c) h->kt[c].collect();
    vanka0 = h->kt[KC_VANKA_APPLY].ms;
    h->t_rebuild.ms = h->t_mg.ms = 0;
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    cudaEventRecord(e0, h->stream);
  }
  stmg_status rs;
  if (h->group) {
    group_enter(h);
    rs = h->precond_fp32() ? newton<float>(h, *group_core_mg<float>(h), t_start, V_prev, U, S)
                           : newton<double>(h, *group_core_mg<double>(h), t_start, V_prev, U, S);
    group_leave(h);
  } else {
    rs = h->precond_fp32() ? newton<float>(h, *h->mg32, t_start, V_prev, U, S)
                           : newton<double>(h, *h->mg64, t_start, V_prev, U, S);
  }
  if (!h->group && (rs == STMG_OK || rs == STMG_ERR_NOT_CONVERGED)) {
    const cudaError_t w = h->precond_fp32() ? h->mg32->check_wait() : h->mg64->check_wait();
    if (w == cudaErrorTimeout) rs = h->fail(STMG_ERR_TIMEOUT, "slab_solve: a bounded wait in the Vanka apply ran out");
    else if (w != cudaSuccess) rs = h->fail(STMG_ERR_CUDA, std::string("slab_solve: ") + cudaGetErrorString(w));
  }
  if (h->timing) {
    cudaEventRecord(e1, h->stream);
    cudaEventSynchronize(e1);
    float tot = 0;
    cudaEventElapsedTime(&tot, e0, e1);
    h->t_rebuild.collect(); h->t_mg.collect();
    for (int c = 0; c < KC_COUNT; ++c) h->kt[c].collect();
    const double tv = h->kt[KC_VANKA_APPLY].ms - vanka0;
    S->t_rebuild = h->t_rebuild.ms * 1e-3;
    S->t_vanka = tv * 1e-3;
    S->t_mg_other = (h->t_mg.ms - tv) * 1e-3;
    S->t_other = (tot - h->t_rebuild.ms - h->t_mg.ms) * 1e-3;
    cudaEventDestroy(e0); cudaEventDestroy(e1);
  }
  return rs;
}

}  // extern "C"
