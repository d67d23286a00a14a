// Host-side reference data for one (d, r, k) level: quadrature rules, 1D bases, time matrices.
//
// Space (Sec. 2.2): velocity Q_{r+1} with Lagrange nodes at the n = r+2 Gauss-Lobatto points
// of [0,1]; quadrature with n_q = r+2 Gauss-Legendre points per direction; pressure P_r^disc
// with the tensor Legendre basis P_i(2x-1) P_j(2y-1) [P_l(2z-1)], i+j(+l) <= r.
// Time (Sec. 3.1 and Appendix A): right Gauss-Radau points of [-1,1] (roots of P_k - P_{k+1}),
// weights exact to degree 2k, the nodal Lagrange basis phi_a and the matrices
//   K_ab = int phi_b' phi_a + phi_b(-1) phi_a(-1),  M = tau/2 diag(omega),  C_a = phi_a(-1).
#pragma once
#include <vector>

namespace stmg {

constexpr int MAXN = 5;      // r + 2 <= 5  (r <= 3)
constexpr int MAXKP1 = 3;    // k + 1 <= 3  (k <= 2)
constexpr int MAXNP = 20;    // C(r+d, d) <= C(6, 3)

// Legendre polynomial P_n and its derivative at x (three-term recurrence).
void legendre(int n, double x, double* p, double* dp);
std::vector<double> gauss_legendre_nodes(int n);            // on [-1,1], ascending
std::vector<double> gauss_legendre_weights(const std::vector<double>& x);
std::vector<double> gauss_lobatto_nodes(int n);             // on [-1,1], ascending
std::vector<double> radau_right_nodes(int k);               // k+1 nodes on [-1,1], last = 1
std::vector<double> exact_weights(const std::vector<double>& x, int degree); // moment fit
double lagrange(const std::vector<double>& nodes, int i, double x);
double lagrange_d(const std::vector<double>& nodes, int i, double x);

struct LevelTables {
  int d, r, k, n, nq, npc;
  // space, on [0,1]
  double gll[MAXN];            // velocity nodes
  double qx[MAXN], qw[MAXN];   // Gauss points / weights (sum 1)
  double B[MAXN][MAXN];        // B[q][j] = l_j(qx_q)      (GLL Lagrange at Gauss points)
  double D[MAXN][MAXN];        // D[q][j] = l_j'(qx_q)
  double Dc[MAXN][MAXN];       // Dc[q][p] = g_p'(qx_q), g = Gauss-point Lagrange basis (collocation)
  double Dend[2][MAXN];        // Dend[s][j] = l_j'(s), s in {0,1}
  double P1[MAXN][4];          // P1[q][i] = P_i(2 qx_q - 1)
  double Pend[2][4];           // Pend[s][i] = P_i(2s - 1)
  int modes[MAXNP][3];
  // time
  double that[MAXKP1], omega[MAXKP1];
  double K[MAXKP1][MAXKP1], C[MAXKP1];
  double phi_mid[MAXKP1];      // phi_a at the slab midpoint (t_hat = 0)
  // Time diagonalisation of the Vanka patch (Sec. 4.3: the spatial core of the surrogate patch
  // is shared by all time nodes).  Omega^{-1} K = Q diag(mu) Q^{-1}, Omega = diag(omega); for a
  // slab of length tau the patch time matrix W^{-1} K (W = tau/2 Omega) has eigenvalues
  // (2/tau) mu and the same Q.  One block per real eigenvalue and one per complex-conjugate pair
  // (represented by its member with Im mu > 0); tnunits = k+1 real units (complex blocks 2).
  int tnblk = 0;
  int tcplx[MAXKP1] = {}, toff[MAXKP1] = {};     // block is complex; first unit of the block
  double tmu_re[MAXKP1] = {}, tmu_im[MAXKP1] = {};
  double tF_re[MAXKP1][MAXKP1] = {}, tF_im[MAXKP1][MAXKP1] = {};   // [block][a]: row of Q^{-1} Omega^{-1}
  double tG_re[MAXKP1][MAXKP1] = {}, tG_im[MAXKP1][MAXKP1] = {};   // [a][block]: Q column, x2 if complex
  void build(int d, int r, int k);
};

}  // namespace stmg
