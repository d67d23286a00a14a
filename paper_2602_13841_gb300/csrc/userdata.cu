// Caller-supplied problem data (STMG_USER): the body force f, the Dirichlet data g and the initial
// velocity v0 of the slab problem (Sec. 2, Problem 2.1; Eq. DefFn, DefLn) given as host callbacks.
//
// The library evaluates f at the volume Gauss points and g at the boundary-face Gauss points of the
// finest mesh, once per slab start time (at the k+1 Radau times t_n^a of the slab), and keeps the
// values in two device tables that the residual kernels read in place of the analytic data of the
// bundled problems (layout: LevelArgs::ftab / gtab).  v0 is evaluated at the velocity nodes.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "../../include/stmg.h"
#include "handle.hpp"
#include "userdata.hpp"

namespace stmg {

// Physical point of the reference point xh of cell cc (multilinear map of the 2^d cell vertices;
// vertices vertex-major, lexicographic with x fastest).
static void host_map(const std::vector<double>& verts, int d, int n, const int* cc, const double* xh, double* x) {
  for (int i = 0; i < d; ++i) x[i] = 0.0;
  for (int c = 0; c < (1 << d); ++c) {
    double wgt = 1.0;
    int64_t v = 0, s = 1;
    for (int l = 0; l < d; ++l) {
      const int b = (c >> l) & 1;
      wgt *= b ? xh[l] : 1.0 - xh[l];
      v += (int64_t)(cc[l] + b) * s;
      s *= (n + 1);
    }
    for (int i = 0; i < d; ++i) x[i] += verts[v * d + i] * wgt;
  }
}

static int64_t ipow64(int64_t b, int e) { int64_t r = 1; for (int i = 0; i < e; ++i) r *= b; return r; }

// Gauss points of the finest level (SoA, d x npts): volume points cell-major (cells
// lexicographic, x fastest) with the N^d points of a cell lexicographic; then the boundary-face
// points, ordered (axis, side, face f, face point p) as in LevelArgs::gtab.
static void user_points(const Handle* h, std::vector<double>& fx, std::vector<double>& gx) {
  const Level& L = h->levels[0];
  const int d = L.d, n = L.n, N = L.r + 2;
  const int64_t ncells = ipow64(n, d), Q = ipow64(N, d), NF = ipow64(N, d - 1), nf = ipow64(n, d - 1);
  const int64_t npf = ncells * Q, npg = (int64_t)d * 2 * nf * NF;
  fx.assign((size_t)d * npf, 0.0);
  gx.assign((size_t)d * npg, 0.0);
  double xh[3] = {0, 0, 0}, x[3];
  int cc[3] = {0, 0, 0};
  for (int64_t cell = 0; cell < ncells; ++cell) {
    int64_t rem = cell;
    for (int l = 0; l < d; ++l) { cc[l] = (int)(rem % n); rem /= n; }
    for (int64_t q = 0; q < Q; ++q) {
      int64_t qr = q;
      for (int l = 0; l < d; ++l) { xh[l] = L.tabs.qx[qr % N]; qr /= N; }
      host_map(h->verts0, d, n, cc, xh, x);
      for (int i = 0; i < d; ++i) fx[(size_t)i * npf + cell * Q + q] = x[i];
    }
  }
  for (int axis = 0; axis < d; ++axis)
    for (int side = 0; side < 2; ++side)
      for (int64_t f = 0; f < nf; ++f) {
        int64_t rem = f;
        for (int l = 0; l < d; ++l) {
          if (l == axis) { cc[l] = side ? n - 1 : 0; continue; }
          cc[l] = (int)(rem % n); rem /= n;
        }
        for (int64_t p = 0; p < NF; ++p) {
          int64_t pr = p;
          for (int l = 0; l < d; ++l) {
            if (l == axis) { xh[l] = (double)side; continue; }
            xh[l] = L.tabs.qx[pr % N]; pr /= N;
          }
          host_map(h->verts0, d, n, cc, xh, x);
          const int64_t idx = ((int64_t)(axis * 2 + side) * nf + f) * NF + p;
          for (int i = 0; i < d; ++i) gx[(size_t)i * npg + idx] = x[i];
        }
      }
}

// Fill the device tables for the slab starting at t0 (no work if they already hold that slab).
cudaError_t refresh_user_data(Handle* h, double t0) {
  if (h->pb.problem != STMG_USER || !h->ftab) return cudaSuccess;
  if (h->user_valid && h->user_t0 == t0) return cudaSuccess;
  const Level& L = h->levels[0];
  const int d = L.d, n = L.n, N = L.r + 2, kp1 = L.k + 1;
  const int64_t ncells = ipow64(n, d), Q = ipow64(N, d), NF = ipow64(N, d - 1), nf = ipow64(n, d - 1);
  const int64_t npf = ncells * Q, npg = (int64_t)d * 2 * nf * NF;
  std::vector<double> out((size_t)d * std::max(npf, npg));
  std::vector<double> ft((size_t)kp1 * d * npf, 0.0), gt((size_t)kp1 * d * npg, 0.0);
  for (int a = 0; a < kp1; ++a) {
    const double ta = t0 + 0.5 * h->pb.tau * (L.tabs.that[a] + 1.0);
    if (h->user_f) {
      std::fill(out.begin(), out.end(), 0.0);
      h->user_f(h->user_ctx, npf, h->user_fx.data(), ta, out.data());
      // ftab[((a ncells + cell) d + c) Q + q] <- out[c npf + cell Q + q]
      for (int64_t cell = 0; cell < ncells; ++cell)
        for (int c = 0; c < d; ++c)
          for (int64_t q = 0; q < Q; ++q)
            ft[(((size_t)a * ncells + cell) * d + c) * Q + q] = out[(size_t)c * npf + cell * Q + q];
    }
    if (h->user_g) {
      std::fill(out.begin(), out.end(), 0.0);
      h->user_g(h->user_ctx, npg, h->user_gx.data(), ta, out.data());
      // gtab[((((a d + axis) 2 + side) nf + f) d + c) NF + p] <- out[c npg + ((axis 2 + side) nf + f) NF + p]
      for (int64_t fs = 0; fs < (int64_t)d * 2 * nf; ++fs)
        for (int c = 0; c < d; ++c)
          for (int64_t p = 0; p < NF; ++p)
            gt[(((size_t)a * d * 2 * nf + fs) * d + c) * NF + p] = out[(size_t)c * npg + fs * NF + p];
    }
  }
  for (double v : ft) if (!std::isfinite(v)) return cudaErrorInvalidValue;
  for (double v : gt) if (!std::isfinite(v)) return cudaErrorInvalidValue;
  try {
    h->upload(h->ftab, ft.data(), ft.size() * sizeof(double));
    h->upload(h->gtab, gt.data(), gt.size() * sizeof(double));
  } catch (const CudaFailure& f) {
    return f.err;
  }
  h->user_t0 = t0;
  h->user_valid = true;
  return cudaSuccess;
}

}  // namespace stmg

using namespace stmg;

extern "C" {

stmg_status stmg_set_data(stmg_handle* hh, stmg_field_fn f, stmg_field_fn g, void* user) {
  if (!hh) return STMG_ERR_ARG;
  Handle* h = reinterpret_cast<Handle*>(hh);
  const Level& L = h->levels[0];
  const int d = L.d, n = L.n, N = L.r + 2, kp1 = L.k + 1;
  const int64_t ncells = ipow64(n, d), Q = ipow64(N, d), NF = ipow64(N, d - 1), nf = ipow64(n, d - 1);
  try {
    if (!h->ftab) {
      h->ftab = (double*)h->dalloc((size_t)kp1 * d * ncells * Q * sizeof(double));
      h->gtab = (double*)h->dalloc((size_t)kp1 * d * 2 * nf * d * NF * sizeof(double));
      user_points(h, h->user_fx, h->user_gx);
    }
  } catch (const std::bad_alloc&) {
    return h->fail(STMG_ERR_OOM, "set_data: no device memory for the data tables");
  }
  h->user_f = f;
  h->user_g = g;
  h->user_ctx = user;
  h->user_valid = false;
  h->prm.problem = STMG_USER;
  h->pb.problem = STMG_USER;
  h->pb.ftab = h->ftab;
  h->pb.gtab = h->gtab;
  // the captured V-cycle bakes the problem parameters into its kernel arguments
  if (h->mg32) h->mg32->drop_graph();
  if (h->mg64) h->mg64->drop_graph();
  return STMG_OK;
}

}  // extern "C"
