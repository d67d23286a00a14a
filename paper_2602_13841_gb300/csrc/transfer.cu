// Grid transfer kernels and their host set-up (see transfer.hpp).
#include <cmath>
#include <vector>

#include "handle.hpp"
#include "transfer.hpp"
#include "counters.hpp"

namespace stmg {

// ---------------------------------------------------------------------------- host set-up
static Csr1D upload_csr(Handle* h, int rows, int cols, const std::vector<std::vector<std::pair<int, double>>>& R) {
  Csr1D c;
  c.rows = rows; c.cols = cols;
  std::vector<int> rp{0}, ci;
  std::vector<double> v;
  std::vector<float> v32;
  for (auto& row : R) {
    for (auto& e : row) { ci.push_back(e.first); v.push_back(e.second); v32.push_back((float)e.second); }
    rp.push_back((int)ci.size());
  }
  c.rowptr = (int*)h->dalloc(rp.size() * sizeof(int));
  c.col = (int*)h->dalloc(ci.size() * sizeof(int));
  c.val64 = (double*)h->dalloc(v.size() * sizeof(double));
  c.val32 = (float*)h->dalloc(v.size() * sizeof(float));
  h->upload(c.rowptr, rp.data(), rp.size() * sizeof(int));
  h->upload(c.col, ci.data(), ci.size() * sizeof(int));
  h->upload(c.val64, v.data(), v.size() * sizeof(double));
  h->upload(c.val32, v32.data(), v32.size() * sizeof(float));
  return c;
}

// rows: value at positions x (in cells of the `n`-cell line) of the global 1D basis of degree r+1
static std::vector<std::vector<std::pair<int, double>>> eval_rows(int n, int r, const std::vector<double>& x) {
  auto g = gauss_lobatto_nodes(r + 2);
  for (auto& v : g) v = 0.5 * (v + 1.0);
  std::vector<std::vector<std::pair<int, double>>> R(x.size());
  for (size_t p = 0; p < x.size(); ++p) {
    int c = (int)std::floor(x[p]);
    if (c > n - 1) c = n - 1;
    if (c < 0) c = 0;
    double xi = x[p] - c;
    for (int j = 0; j < r + 2; ++j) {
      double v = lagrange(g, j, xi);
      if (std::fabs(v) > 1e-14) R[p].push_back({c * (r + 1) + j, v});
    }
  }
  return R;
}

static std::vector<double> node_positions(int n, int r, double scale) {
  auto g = gauss_lobatto_nodes(r + 2);
  std::vector<double> x;
  for (int c = 0; c < n; ++c)
    for (int i = 0; i <= r; ++i) x.push_back((c + 0.5 * (g[i] + 1.0)) * scale);
  x.push_back(n * scale);
  return x;
}

void build_transfer(Handle* h, Transfer& tr, const Level& f, const Level& c, size_t esize, int nb) {
  tr.fine = &f; tr.coarse = &c;
  const double cf = (double)c.n / f.n;
  auto R = eval_rows(c.n, c.r, node_positions(f.n, f.r, cf));
  tr.P1 = upload_csr(h, f.N1, c.N1, R);
  std::vector<std::vector<std::pair<int, double>>> RT(c.N1);
  for (int i = 0; i < (int)R.size(); ++i)
    for (auto& e : R[i]) RT[e.first].push_back({i, e.second});
  tr.P1T = upload_csr(h, c.N1, f.N1, RT);
  tr.I1 = upload_csr(h, c.N1, f.N1, eval_rows(f.n, f.r, node_positions(c.n, c.r, 1.0 / cf)));
  // time
  auto tf = radau_right_nodes(f.k), tc = radau_right_nodes(c.k);
  for (int i = 0; i <= f.k; ++i)
    for (int j = 0; j <= c.k; ++j) {
      tr.E[i][j] = (c.k == 0) ? 1.0 : lagrange(tc, j, tf[i]);
      tr.Et[j][i] = (f.k == 0) ? 1.0 : lagrange(tf, i, tc[j]);
    }
  // pressure child expansions: T1[b][i][j] = coeff of P_j(2x-1) in P_i(2 (b+x)/2 - 1)
  tr.ratio = f.n / c.n;
  tr.ntypes = (tr.ratio == 2) ? (1 << f.d) : 1;
  const int rr = f.r > c.r ? f.r : c.r;
  auto gx = gauss_legendre_nodes(rr + 2);
  auto gw = gauss_legendre_weights(gx);
  double T1[2][4][4] = {};
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i <= rr; ++i)
      for (int j = 0; j <= rr; ++j) {
        double s = 0;
        for (size_t q = 0; q < gx.size(); ++q) {
          double x = 0.5 * (gx[q] + 1.0), w = 0.5 * gw[q];
          double pi, dpi, pj, dpj;
          legendre(i, 2.0 * (0.5 * (b + x)) - 1.0, &pi, &dpi);
          legendre(j, 2.0 * x - 1.0, &pj, &dpj);
          s += w * pi * pj;
        }
        T1[b][i][j] = s * (2 * j + 1);
      }
  const int npf = f.npc, npc = c.npc;
  std::vector<double> PT(tr.ntypes * npf * npc, 0.0);
  for (int t = 0; t < tr.ntypes; ++t)
    for (int mf = 0; mf < npf; ++mf)
      for (int mc = 0; mc < npc; ++mc) {
        double v;
        if (tr.ratio == 1) {
          v = 1.0;
          for (int l = 0; l < f.d; ++l) if (f.tabs.modes[mf][l] != c.tabs.modes[mc][l]) v = 0.0;
        } else {
          v = 1.0;
          for (int l = 0; l < f.d; ++l) v *= T1[(t >> l) & 1][c.tabs.modes[mc][l]][f.tabs.modes[mf][l]];
        }
        PT[(t * npf + mf) * npc + mc] = v;
      }
  std::vector<float> PT32(PT.begin(), PT.end());
  tr.PT64 = (double*)h->dalloc(PT.size() * sizeof(double));
  tr.PT32 = (float*)h->dalloc(PT.size() * sizeof(float));
  h->upload(tr.PT64, PT.data(), PT.size() * sizeof(double));
  h->upload(tr.PT32, PT32.data(), PT32.size() * sizeof(float));
  // scratch: largest intermediate = (max k + 1) * d * max(N1f^d, ...) or the pressure part
  int64_t big = (int64_t)(f.k + 1) * f.Nv;
  int64_t pbig = (int64_t)(f.k + 1) * f.Np;
  if (pbig > big) big = pbig;
  tr.nb = nb;
  tr.scr = big;
  tr.tmpA = h->dalloc((size_t)nb * big * esize);
  tr.tmpB = h->dalloc((size_t)nb * big * esize);
  tr.tmpC = h->dalloc((size_t)nb * big * esize);
}

// ---------------------------------------------------------------------------- kernels
// out[b][o][i][p] = sum_k val[k] in[b][o][col[k]][p], k in row i; arrays of `batch` contiguous
// blocks (strides sin / sout), axis extent nin -> nout, `inner` = product of faster axes.
template <typename T>
__global__ void k_axis(const T* __restrict__ in, T* __restrict__ out, int nin, int nout, int64_t inner,
                       int64_t outer, int64_t sin, int64_t sout, const int* __restrict__ rowptr,
                       const int* __restrict__ col, const T* __restrict__ val, int64_t zin, int64_t zout) {
  const int b = blockIdx.y;
  const int64_t total = outer * nout * inner;
  in += b * sin + blockIdx.z * zin;           // blockIdx.z: independent slot
  out += b * sout + blockIdx.z * zout;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = idx % inner;
    int64_t rest = idx / inner;
    int i = (int)(rest % nout);
    int64_t o = rest / nout;
    T acc = 0;
    for (int kk = rowptr[i]; kk < rowptr[i + 1]; ++kk) acc += val[kk] * in[(o * nin + col[kk]) * inner + p];
    out[idx] = acc;
  }
}

// out[a_out][i] = sum_{a_in} M[a_out][a_in] in[a_in][i]   (arrays of length L)
struct Mat3 { double m[MAXKP1][MAXKP1]; };
template <typename T>
__global__ void k_timemix(const T* __restrict__ in, T* __restrict__ out, int64_t L, int nin, int nout,
                          int64_t sin, int64_t sout, Mat3 M, int64_t zin, int64_t zout) {
  in += blockIdx.y * zin;                     // blockIdx.y: independent slot
  out += blockIdx.y * zout;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x) {
    T v[MAXKP1];
    for (int a = 0; a < nin; ++a) v[a] = in[a * sin + i];
    for (int a = 0; a < nout; ++a) {
      T acc = 0;
      for (int b = 0; b < nin; ++b) acc += (T)M.m[a][b] * v[b];
      out[a * sout + i] = acc;
    }
  }
}

// Pressure prolongation: fine cell cf, mode mf  <-  coarse cell, all coarse modes (per time node)
template <typename T, int D>
__global__ void k_pprolong(const T* __restrict__ in, T* __restrict__ out, int nf, int ratio, int npf, int npc,
                           const T* __restrict__ PT, int64_t sin, int64_t sout, int64_t zin, int64_t zout) {
  const int b = blockIdx.y;
  in += b * sin + blockIdx.z * zin; out += b * sout + blockIdx.z * zout;
  int64_t ncf = 1;
  for (int l = 0; l < D; ++l) ncf *= nf;
  const int nc = nf / ratio;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < ncf * npf;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int mf = (int)(idx % npf);
    int64_t cf = idx / npf, rem = cf, cc = 0, s = 1;
    int type = 0;
    for (int l = 0; l < D; ++l) {
      int x = (int)(rem % nf); rem /= nf;
      cc += (int64_t)(x / ratio) * s; s *= nc;
      if (ratio == 2) type |= (x & 1) << l;
    }
    const T* row = PT + ((int64_t)type * npf + mf) * npc;
    T acc = 0;
    for (int mc = 0; mc < npc; ++mc) acc += row[mc] * in[cc * npc + mc];
    out[idx] = acc;
  }
}

// Pressure restriction (transpose): coarse cell, mode mc  <-  its fine cells, all fine modes
template <typename T, int D>
__global__ void k_prestrict(const T* __restrict__ in, T* __restrict__ out, int nf, int ratio, int npf, int npc,
                            const T* __restrict__ PT, int64_t sin, int64_t sout, int64_t zin, int64_t zout) {
  const int b = blockIdx.y;
  in += b * sin + blockIdx.z * zin; out += b * sout + blockIdx.z * zout;
  const int nc = nf / ratio;
  int64_t ncc = 1;
  for (int l = 0; l < D; ++l) ncc *= nc;
  const int nchild = (ratio == 2) ? (1 << D) : 1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < ncc * npc;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int mc = (int)(idx % npc);
    int64_t cc = idx / npc;
    int cm[3] = {0, 0, 0};
    int64_t rem = cc;
    for (int l = 0; l < D; ++l) { cm[l] = (int)(rem % nc); rem /= nc; }
    T acc = 0;
    for (int ch = 0; ch < nchild; ++ch) {
      int64_t cf = 0, s = 1;
      for (int l = 0; l < D; ++l) { cf += (int64_t)(cm[l] * ratio + ((ch >> l) & 1) * (ratio - 1)) * s; s *= nf; }
      const T* P = PT + (int64_t)ch * npf * npc;
      for (int mf = 0; mf < npf; ++mf) acc += P[mf * npc + mc] * in[cf * npf + mf];
    }
    out[idx] = acc;
  }
}

static inline int grid1(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  return (int)(g < 1 ? 1 : g);
}

template <typename T> static const T* vals(const Csr1D& c);
template <> const double* vals<double>(const Csr1D& c) { return c.val64; }
template <> const float* vals<float>(const Csr1D& c) { return c.val32; }
template <typename T> static const T* ptab(const Transfer& t);
template <> const double* ptab<double>(const Transfer& t) { return t.PT64; }
template <> const float* ptab<float>(const Transfer& t) { return t.PT32; }

// Apply a 1D operator along every axis to `batch` arrays of nin^d entries -> nout^d entries.
// `slots` independent inputs at in + j * zin (outputs out + j * zout, scratch t + j * zt).
template <typename T>
static cudaError_t tensor_apply(const Csr1D& op, int d, int nin, int nout, int batch, const T* in, T* out,
                                T* t1, T* t2, cudaStream_t s, int slots = 1, int64_t zin = 0, int64_t zout = 0,
                                int64_t zt = 0) {
  int64_t ext[3] = {nin, nin, nin};
  const T* src = in;
  int64_t sin = 1;
  for (int l = 0; l < d; ++l) sin *= nin;
  for (int ax = 0; ax < d; ++ax) {
    int64_t inner = 1, outer = 1;
    for (int l = 0; l < ax; ++l) inner *= ext[l];
    for (int l = ax + 1; l < d; ++l) outer *= ext[l];
    int64_t sout = 1;
    for (int l = 0; l < d; ++l) sout *= (l == ax ? nout : ext[l]);
    T* dst = (ax == d - 1) ? out : ((ax % 2 == 0) ? t1 : t2);
    int64_t sdst = (ax == d - 1) ? 0 : sout;
    // the final pass writes with the caller's stride (= nout^d)
    if (ax == d - 1) sdst = sout;
    dim3 grid(grid1(outer * nout * inner), batch, slots);
    const int64_t zs = (ax == 0) ? zin : zt, zd = (ax == d - 1) ? zout : zt;
    k_axis<T><<<grid, 256, 0, s>>>(src, dst, (int)ext[ax], nout, inner, outer, sin, sdst, op.rowptr, op.col,
                                   vals<T>(op), zs, zd);
    note_launch();
    ext[ax] = nout;
    src = dst;
    sin = sdst;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t Transfer::prolong(const T* xc, T* xf, cudaStream_t s, int slots) const {
  const Level& f = *fine; const Level& c = *coarse;
  if (slots < 1 || slots > nb) return cudaErrorInvalidValue;
  T* A = (T*)tmpA; T* B = (T*)tmpB; T* C = (T*)tmpC;
  const int d = f.d;
  // velocity: space at coarse time nodes -> C, then time mix into xf
  cudaError_t e = tensor_apply<T>(P1, d, c.N1, f.N1, (c.k + 1) * d, xc, C, A, B, s, slots, c.Nst, scr, scr);
  if (e != cudaSuccess) return e;
  Mat3 M{};
  for (int a = 0; a <= f.k; ++a) for (int b = 0; b <= c.k; ++b) M.m[a][b] = E[a][b];
  k_timemix<T><<<dim3(grid1(f.Nv), slots), 256, 0, s>>>(C, xf, f.Nv, c.k + 1, f.k + 1, f.Nv, f.Nv, M, scr, f.Nst);
  note_launch();
  // pressure
  const T* pc = xc + (int64_t)(c.k + 1) * c.Nv;
  T* pf = xf + (int64_t)(f.k + 1) * f.Nv;
  int64_t ncf = f.Np / f.npc;
  dim3 g(grid1(ncf * f.npc), c.k + 1, slots);
  if (d == 2) k_pprolong<T, 2><<<g, 256, 0, s>>>(pc, C, f.n, ratio, f.npc, c.npc, ptab<T>(*this), c.Np, f.Np, c.Nst, scr);
  else k_pprolong<T, 3><<<g, 256, 0, s>>>(pc, C, f.n, ratio, f.npc, c.npc, ptab<T>(*this), c.Np, f.Np, c.Nst, scr);
  note_launch();
  k_timemix<T><<<dim3(grid1(f.Np), slots), 256, 0, s>>>(C, pf, f.Np, c.k + 1, f.k + 1, f.Np, f.Np, M, scr, f.Nst);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t Transfer::restrict_(const T* xf, T* xc, cudaStream_t s, int slots) const {
  const Level& f = *fine; const Level& c = *coarse;
  if (slots < 1 || slots > nb) return cudaErrorInvalidValue;
  T* A = (T*)tmpA; T* B = (T*)tmpB; T* C = (T*)tmpC;
  const int d = f.d;
  Mat3 M{};
  for (int a = 0; a <= c.k; ++a) for (int b = 0; b <= f.k; ++b) M.m[a][b] = E[b][a];   // E^T
  k_timemix<T><<<dim3(grid1(f.Nv), slots), 256, 0, s>>>(xf, C, f.Nv, f.k + 1, c.k + 1, f.Nv, f.Nv, M, f.Nst, scr);
  note_launch();
  cudaError_t e = tensor_apply<T>(P1T, d, f.N1, c.N1, (c.k + 1) * d, C, xc, A, B, s, slots, scr, c.Nst, scr);
  if (e != cudaSuccess) return e;
  const T* pf = xf + (int64_t)(f.k + 1) * f.Nv;
  T* pc = xc + (int64_t)(c.k + 1) * c.Nv;
  k_timemix<T><<<dim3(grid1(f.Np), slots), 256, 0, s>>>(pf, C, f.Np, f.k + 1, c.k + 1, f.Np, f.Np, M, f.Nst, scr);
  note_launch();
  int64_t ncc = c.Np / c.npc;
  dim3 g(grid1(ncc * c.npc), c.k + 1, slots);
  if (d == 2) k_prestrict<T, 2><<<g, 256, 0, s>>>(C, pc, f.n, ratio, f.npc, c.npc, ptab<T>(*this), f.Np, c.Np, scr, c.Nst);
  else k_prestrict<T, 3><<<g, 256, 0, s>>>(C, pc, f.n, ratio, f.npc, c.npc, ptab<T>(*this), f.Np, c.Np, scr, c.Nst);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t Transfer::interp_state(const T* Vf, T* Vc, cudaStream_t s) const {
  const Level& f = *fine; const Level& c = *coarse;
  T* A = (T*)tmpA; T* B = (T*)tmpB; T* C = (T*)tmpC;
  Mat3 M{};
  for (int a = 0; a <= c.k; ++a) for (int b = 0; b <= f.k; ++b) M.m[a][b] = Et[a][b];
  k_timemix<T><<<grid1(f.Nv), 256, 0, s>>>(Vf, C, f.Nv, f.k + 1, c.k + 1, f.Nv, f.Nv, M, 0, 0);
  note_launch();
  return tensor_apply<T>(I1, f.d, f.N1, c.N1, (c.k + 1) * f.d, C, Vc, A, B, s);
}

template cudaError_t Transfer::prolong<float>(const float*, float*, cudaStream_t, int) const;
template cudaError_t Transfer::prolong<double>(const double*, double*, cudaStream_t, int) const;
template cudaError_t Transfer::restrict_<float>(const float*, float*, cudaStream_t, int) const;
template cudaError_t Transfer::restrict_<double>(const double*, double*, cudaStream_t, int) const;
template cudaError_t Transfer::interp_state<float>(const float*, float*, cudaStream_t) const;
template cudaError_t Transfer::interp_state<double>(const double*, double*, cudaStream_t) const;

}  // namespace stmg
