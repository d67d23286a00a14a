// Host reference data (see refdata.hpp).  Roots are bracketed on a fine grid and refined by
// bisection, which is robust for the low degrees used here (<= 6).
#include "refdata.hpp"

#include <algorithm>
#include <cmath>
#include <complex>
#include <utility>
#include <stdexcept>

namespace stmg {

void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int m = 2; m <= n; ++m) {
    double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) / m;
    double d2 = d0 + (2.0 * m - 1.0) * p1;   // P'_m = P'_{m-2} + (2m-1) P_{m-1}
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *p = p1; *dp = d1;
}

template <class F>
static std::vector<double> roots_in(F f, double a, double b, int expect) {
  std::vector<double> out;
  const int M = 20000;
  double xa = a, fa = f(a);
  for (int i = 1; i <= M; ++i) {
    double xb = a + (b - a) * i / M, fb = f(xb);
    if (fa == 0.0) { out.push_back(xa); }
    else if (fa * fb < 0.0) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi), fm = f(mid);
        if (fm == 0.0) { lo = hi = mid; break; }
        if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      out.push_back(0.5 * (lo + hi));
    }
    xa = xb; fa = fb;
  }
  if ((int)out.size() != expect) throw std::runtime_error("root bracketing failed");
  return out;
}

std::vector<double> gauss_legendre_nodes(int n) {
  return roots_in([n](double x) { double p, dp; legendre(n, x, &p, &dp); return p; },
                  -1.0 + 1e-9, 1.0 - 1e-9, n);
}

std::vector<double> exact_weights(const std::vector<double>& x, int degree) {
  // Solve sum_i w_i x_i^p = int_{-1}^{1} t^p dt for p = 0..n-1 (Gaussian elimination).
  int n = (int)x.size();
  (void)degree;
  std::vector<double> A(n * (n + 1));
  for (int p = 0; p < n; ++p) {
    for (int i = 0; i < n; ++i) A[p * (n + 1) + i] = std::pow(x[i], p);
    A[p * (n + 1) + n] = (1.0 - std::pow(-1.0, p + 1)) / (p + 1);
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * (n + 1) + c]) > std::fabs(A[piv * (n + 1) + c])) piv = r;
    for (int j = 0; j <= n; ++j) std::swap(A[c * (n + 1) + j], A[piv * (n + 1) + j]);
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * (n + 1) + c] / A[c * (n + 1) + c];
      for (int j = c; j <= n; ++j) A[r * (n + 1) + j] -= f * A[c * (n + 1) + j];
    }
  }
  std::vector<double> w(n);
  for (int i = 0; i < n; ++i) w[i] = A[i * (n + 1) + n] / A[i * (n + 1) + i];
  return w;
}

std::vector<double> gauss_legendre_weights(const std::vector<double>& x) {
  return exact_weights(x, 2 * (int)x.size() - 1);
}

std::vector<double> gauss_lobatto_nodes(int n) {
  std::vector<double> x{-1.0};
  if (n > 2) {
    auto in = roots_in([n](double t) { double p, dp; legendre(n - 1, t, &p, &dp); return dp; },
                       -1.0 + 1e-9, 1.0 - 1e-9, n - 2);
    x.insert(x.end(), in.begin(), in.end());
  }
  x.push_back(1.0);
  return x;
}

std::vector<double> radau_right_nodes(int k) {
  if (k == 0) return {1.0};
  auto in = roots_in([k](double t) {
    double pk, dk, pk1, dk1;
    legendre(k, t, &pk, &dk);
    legendre(k + 1, t, &pk1, &dk1);
    return pk - pk1;
  }, -1.0 + 1e-9, 1.0 - 1e-7, k);
  in.push_back(1.0);
  return in;
}

double lagrange(const std::vector<double>& nodes, int i, double x) {
  double v = 1.0;
  for (int j = 0; j < (int)nodes.size(); ++j)
    if (j != i) v *= (x - nodes[j]) / (nodes[i] - nodes[j]);
  return v;
}

double lagrange_d(const std::vector<double>& nodes, int i, double x) {
  double s = 0.0;
  int n = (int)nodes.size();
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    double t = 1.0 / (nodes[i] - nodes[m]);
    for (int j = 0; j < n; ++j)
      if (j != i && j != m) t *= (x - nodes[j]) / (nodes[i] - nodes[j]);
    s += t;
  }
  return s;
}

using cplx = std::complex<double>;

// Roots of z^3 + a2 z^2 + a1 z + a0 (Durand-Kerner iteration, then Newton polishing).
static void cubic_roots(cplx a2, cplx a1, cplx a0, cplx z[3]) {
  auto f = [&](cplx x) { return ((x + a2) * x + a1) * x + a0; };
  auto df = [&](cplx x) { return (3.0 * x + 2.0 * a2) * x + a1; };
  const cplx seed(0.4, 0.9);
  z[0] = 1.0; z[1] = seed; z[2] = seed * seed;
  for (int it = 0; it < 500; ++it)
    for (int i = 0; i < 3; ++i) {
      cplx den = 1.0;
      for (int j = 0; j < 3; ++j) if (j != i) den *= (z[i] - z[j]);
      z[i] -= f(z[i]) / den;
    }
  for (int i = 0; i < 3; ++i)
    for (int it = 0; it < 3; ++it) { cplx g = df(z[i]); if (std::abs(g) > 0) z[i] -= f(z[i]) / g; }
}

// Eigen-decomposition of the (k+1) x (k+1) matrix P = Omega^{-1} K.  Its eigenvalues are
// distinct: k = 0 one real, k = 1 one conjugate pair, k = 2 one pair and one real.
static void time_eigen(LevelTables& T) {
  const int n = T.k + 1;
  double P[3][3] = {};
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) P[a][b] = T.K[a][b] / T.omega[a];
  cplx lam[3], Q[3][3];
  if (n == 1) {
    lam[0] = P[0][0]; Q[0][0] = 1.0;
  } else if (n == 2) {
    const double tr = P[0][0] + P[1][1], det = P[0][0] * P[1][1] - P[0][1] * P[1][0];
    const cplx sq = std::sqrt(cplx(0.25 * tr * tr - det, 0.0));
    lam[0] = 0.5 * tr + sq; lam[1] = 0.5 * tr - sq;
    for (int e = 0; e < 2; ++e) {
      cplx v0 = P[0][1], v1 = lam[e] - P[0][0];
      if (std::abs(v0) + std::abs(v1) < 1e-14) { v0 = lam[e] - P[1][1]; v1 = P[1][0]; }
      const double nv = std::sqrt(std::norm(v0) + std::norm(v1));
      Q[0][e] = v0 / nv; Q[1][e] = v1 / nv;
    }
  } else {
    const double tr = P[0][0] + P[1][1] + P[2][2];
    const double m2 = P[0][0] * P[1][1] - P[0][1] * P[1][0] + P[0][0] * P[2][2] - P[0][2] * P[2][0] +
                      P[1][1] * P[2][2] - P[1][2] * P[2][1];
    const double det = P[0][0] * (P[1][1] * P[2][2] - P[1][2] * P[2][1]) -
                       P[0][1] * (P[1][0] * P[2][2] - P[1][2] * P[2][0]) +
                       P[0][2] * (P[1][0] * P[2][1] - P[1][1] * P[2][0]);
    cubic_roots(-tr, m2, -det, lam);
    for (int e = 0; e < 3; ++e) {
      // null vector of P - lam I: the largest cross product of two of its rows
      cplx R[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) R[a][b] = P[a][b] - (a == b ? lam[e] : cplx(0.0));
      cplx best[3]; double bn = -1;
      const int pr[3][2] = {{0, 1}, {0, 2}, {1, 2}};
      for (auto& q : pr) {
        const cplx* u = R[q[0]]; const cplx* v = R[q[1]];
        cplx c[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        const double nc = std::norm(c[0]) + std::norm(c[1]) + std::norm(c[2]);
        if (nc > bn) { bn = nc; best[0] = c[0]; best[1] = c[1]; best[2] = c[2]; }
      }
      const double nv = std::sqrt(bn);
      for (int a = 0; a < 3; ++a) Q[a][e] = best[a] / nv;
    }
  }
  // real eigenvalues get real eigenvectors; a conjugate partner gets the conjugate column
  bool used[3] = {false, false, false};
  int blk_of[3] = {-1, -1, -1};
  T.tnblk = 0;
  int unit = 0;
  for (int e = 0; e < n; ++e) {
    if (used[e]) continue;
    const double scale = std::max(1.0, std::abs(lam[e]));
    const bool real = std::abs(lam[e].imag()) <= 1e-10 * scale;
    const int b = T.tnblk++;
    used[e] = true;
    if (real) {
      lam[e] = lam[e].real();
      double nv = 0;
      for (int a = 0; a < n; ++a) nv += Q[a][e].real() * Q[a][e].real();
      // a real null vector is a complex multiple of its real part (or imaginary part)
      if (nv < 1e-20) for (int a = 0; a < n; ++a) Q[a][e] = Q[a][e].imag();
      else for (int a = 0; a < n; ++a) Q[a][e] = Q[a][e].real();
      nv = 0;
      for (int a = 0; a < n; ++a) nv += std::norm(Q[a][e]);
      for (int a = 0; a < n; ++a) Q[a][e] /= std::sqrt(nv);
      T.tcplx[b] = 0; T.toff[b] = unit; unit += 1;
      blk_of[e] = b;
    } else {
      int f = -1;
      for (int g = 0; g < n; ++g)
        if (!used[g] && std::abs(lam[g] - std::conj(lam[e])) <= 1e-8 * scale) { f = g; break; }
      if (f < 0) throw std::runtime_error("time matrix: unpaired complex eigenvalue");
      used[f] = true;
      const int rep = lam[e].imag() > 0 ? e : f, par = rep == e ? f : e;
      lam[par] = std::conj(lam[rep]);
      for (int a = 0; a < n; ++a) Q[a][par] = std::conj(Q[a][rep]);
      T.tcplx[b] = 1; T.toff[b] = unit; unit += 2;
      blk_of[rep] = b;
    }
  }
  // Q^{-1} by Gauss-Jordan with partial pivoting (n <= 3)
  cplx A[3][6];
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < 2 * n; ++b) A[a][b] = b < n ? Q[a][b] : cplx(b - n == a ? 1.0 : 0.0);
  for (int p = 0; p < n; ++p) {
    int piv = p;
    for (int a = p + 1; a < n; ++a) if (std::abs(A[a][p]) > std::abs(A[piv][p])) piv = a;
    if (std::abs(A[piv][p]) < 1e-14) throw std::runtime_error("time matrix: singular eigenvectors");
    for (int b = 0; b < 2 * n; ++b) std::swap(A[p][b], A[piv][b]);
    const cplx inv = 1.0 / A[p][p];
    for (int b = 0; b < 2 * n; ++b) A[p][b] *= inv;
    for (int a = 0; a < n; ++a)
      if (a != p) {
        const cplx f = A[a][p];
        for (int b = 0; b < 2 * n; ++b) A[a][b] -= f * A[p][b];
      }
  }
  for (int e = 0; e < n; ++e) {
    const int b = blk_of[e];
    if (b < 0) continue;
    T.tmu_re[b] = lam[e].real();
    T.tmu_im[b] = T.tcplx[b] ? lam[e].imag() : 0.0;
    const double two = T.tcplx[b] ? 2.0 : 1.0;
    for (int a = 0; a < n; ++a) {
      const cplx f = A[e][n + a] / T.omega[a];
      T.tF_re[b][a] = f.real();
      T.tF_im[b][a] = T.tcplx[b] ? f.imag() : 0.0;
      T.tG_re[a][b] = two * Q[a][e].real();
      T.tG_im[a][b] = T.tcplx[b] ? two * Q[a][e].imag() : 0.0;
    }
  }
}

void LevelTables::build(int d_, int r_, int k_) {
  d = d_; r = r_; k = k_;
  n = r + 2; nq = r + 2;
  if (n > MAXN || k + 1 > MAXKP1 || d < 2 || d > 3) throw std::runtime_error("unsupported level");
  auto gl = gauss_lobatto_nodes(n);
  auto gx = gauss_legendre_nodes(nq);
  auto gw = gauss_legendre_weights(gx);
  std::vector<double> g01(n), q01(nq);
  for (int i = 0; i < n; ++i) { g01[i] = 0.5 * (gl[i] + 1.0); gll[i] = g01[i]; }
  for (int q = 0; q < nq; ++q) { q01[q] = 0.5 * (gx[q] + 1.0); qx[q] = q01[q]; qw[q] = 0.5 * gw[q]; }
  for (int q = 0; q < nq; ++q)
    for (int j = 0; j < n; ++j) {
      B[q][j] = lagrange(g01, j, q01[q]);
      D[q][j] = lagrange_d(g01, j, q01[q]);
    }
  for (int q = 0; q < nq; ++q)
    for (int p = 0; p < nq; ++p) Dc[q][p] = lagrange_d(q01, p, q01[q]);
  for (int s = 0; s < 2; ++s)
    for (int j = 0; j < n; ++j) Dend[s][j] = lagrange_d(g01, j, (double)s);
  for (int q = 0; q < nq; ++q)
    for (int i = 0; i <= r; ++i) { double p, dp; legendre(i, 2.0 * q01[q] - 1.0, &p, &dp); P1[q][i] = p; }
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i <= r; ++i) { double p, dp; legendre(i, 2.0 * s - 1.0, &p, &dp); Pend[s][i] = p; }
  // pressure modes: total degree, then ascending degree of the last coordinate
  npc = 0;
  for (int s = 0; s <= r; ++s) {
    if (d == 2) {
      for (int j = 0; j <= s; ++j) { modes[npc][0] = s - j; modes[npc][1] = j; modes[npc][2] = 0; ++npc; }
    } else {
      for (int l = 0; l <= s; ++l)
        for (int j = 0; j <= s - l; ++j) {
          modes[npc][0] = s - j - l; modes[npc][1] = j; modes[npc][2] = l; ++npc;
        }
    }
  }
  // time
  auto tn = radau_right_nodes(k);
  auto tw = exact_weights(tn, 2 * k);
  for (int a = 0; a <= k; ++a) { that[a] = tn[a]; omega[a] = tw[a]; }
  auto gt = gauss_legendre_nodes(k + 3);
  auto gtw = gauss_legendre_weights(gt);
  for (int a = 0; a <= k; ++a) {
    C[a] = (k == 0) ? 1.0 : lagrange(tn, a, -1.0);
    phi_mid[a] = (k == 0) ? 1.0 : lagrange(tn, a, 0.0);
  }
  for (int a = 0; a <= k; ++a)
    for (int b = 0; b <= k; ++b) {
      double s = 0.0;
      if (k > 0)
        for (int q = 0; q < (int)gt.size(); ++q)
          s += gtw[q] * lagrange_d(tn, b, gt[q]) * lagrange(tn, a, gt[q]);
      K[a][b] = s + C[a] * C[b];
    }
  time_eigen(*this);
}

}  // namespace stmg
