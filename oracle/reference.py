"""Reference data: quadrature rules, 1D bases, temporal matrices (oracle; test infrastructure).

Sources in the paper:
  * right-sided (k+1)-point Gauss-Radau rule on [-1,1], exact to degree 2k, last node = +1
    (Sec. 3.1, Eq. (GF));
  * local Lagrange basis in time at the Radau nodes (Eq. BasYk);
  * time matrices K^tau, M^tau, C^tau (Appendix A, Eq. DefKMC);
  * velocity space Q_{r+1}, pressure space mapped P_r^disc (Sec. 2.2, Def. VKQK).
Readings where the paper is silent: velocity nodes are Gauss-Lobatto-Legendre points,
spatial quadrature is (r+2)-point Gauss-Legendre per direction, and the pressure basis is
the tensor Legendre basis L_i(x)L_j(y)[L_l(z)] on [0,1]^d with total degree <= r.
"""
import itertools
import math

import numpy as np
from numpy.polynomial import legendre as npleg


# ----------------------------------------------------------------------------- 1D rules
def gauss_legendre_01(n):
    """n-point Gauss-Legendre rule mapped to [0,1] (library routine; weights sum to 1)."""
    x, w = npleg.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_lobatto_01(n):
    """n-point Gauss-Lobatto-Legendre nodes on [0,1]: the end points and the roots of P'_{n-1}."""
    assert n >= 2
    if n == 2:
        x = np.array([-1.0, 1.0])
    else:
        c = np.zeros(n)
        c[n - 1] = 1.0
        inner = np.sort(np.real(npleg.legroots(npleg.legder(c))))
        x = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (x + 1.0)


def radau_right(k):
    """Right-sided (k+1)-point Gauss-Radau rule on [-1,1] (Sec. 3.1, Eq. GF).

    The nodes are the roots of P_k - P_{k+1} (they include +1); the weights make the rule
    exact for all polynomials of degree <= 2k (moment equations solved by a linear solve).
    """
    if k == 0:
        return np.array([1.0]), np.array([2.0])
    c = np.zeros(k + 2)
    c[k] = 1.0
    c[k + 1] = -1.0
    t = np.sort(np.real(npleg.legroots(c)))
    t[-1] = 1.0
    V = np.array([t ** p for p in range(k + 1)])
    mom = np.array([(1.0 - (-1.0) ** (p + 1)) / (p + 1) for p in range(k + 1)])
    w = np.linalg.solve(V, mom)
    return t, w


# ----------------------------------------------------------------------------- 1D bases
def lagrange_eval(nodes, x):
    """Values L[p, i] = l_i(x_p) of the Lagrange polynomials on `nodes` (product formula)."""
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    n = len(nodes)
    L = np.ones((len(x), n))
    for i in range(n):
        for j in range(n):
            if j != i:
                L[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
    return L


def lagrange_deriv(nodes, x):
    """Derivatives D[p, i] = l_i'(x_p) (product rule on the product formula)."""
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j != i and j != m:
                    term *= (x - nodes[j]) / (nodes[i] - nodes[j])
            D[:, i] += term
    return D


def legendre01(deg, x):
    """Shifted Legendre values P_i(2x-1), i = 0..deg, as array [len(x), deg+1]."""
    x = np.atleast_1d(np.asarray(x, float))
    out = np.zeros((len(x), deg + 1))
    for i in range(deg + 1):
        c = np.zeros(i + 1)
        c[i] = 1.0
        out[:, i] = npleg.legval(2.0 * x - 1.0, c)
    return out


def legendre01_deriv(deg, x):
    """Derivatives d/dx P_i(2x-1) = 2 P_i'(2x-1)."""
    x = np.atleast_1d(np.asarray(x, float))
    out = np.zeros((len(x), deg + 1))
    for i in range(deg + 1):
        c = np.zeros(i + 1)
        c[i] = 1.0
        out[:, i] = 2.0 * npleg.legval(2.0 * x - 1.0, npleg.legder(c)) if i > 0 else 0.0
    return out


def pressure_modes(r, d):
    """Multi-indices of the P_r^disc tensor Legendre basis, ordered by total degree, then by
    ascending degree of the last coordinate, ..., x-degree last (reading of Def. VKQK)."""
    modes = []
    for s in range(r + 1):
        if d == 2:
            for j in range(s + 1):
                modes.append((s - j, j))
        else:
            for l in range(s + 1):
                for j in range(s - l + 1):
                    modes.append((s - j - l, j, l))
    assert len(modes) == math.comb(r + d, d)
    return modes


# ----------------------------------------------------------------------------- time
class TimeData:
    """DG(k) in time on a slab of length tau (Sec. 3.1 and Appendix A, Eq. DefKMC).

    phi_a are the Lagrange polynomials at the right Radau nodes t_hat_a; on the slab
    t = t_{n-1} + tau (t_hat + 1)/2.
      K_ab = int phi_b' phi_a dt + phi_b(t_{n-1}^+) phi_a(t_{n-1}^+)     (tau-independent)
      M_ab = int phi_b phi_a dt  (diagonal, = w_a = tau/2 omega_hat_a by Radau exactness)
      C_a  = phi_a(t_{n-1}^+)   (jump coupling with the last node of the previous slab)
    """

    def __init__(self, k, tau):
        self.k = k
        self.tau = tau
        self.that, self.omega = radau_right(k)
        nodes = self.that
        xg, wg = npleg.leggauss(k + 3)                      # exact for degree 2k+5
        if k == 0:
            phi = np.ones((len(xg), 1))
            dphi = np.zeros((len(xg), 1))
            phim1 = np.ones(1)
        else:
            phi = lagrange_eval(nodes, xg)
            dphi = lagrange_deriv(nodes, xg)
            phim1 = lagrange_eval(nodes, [-1.0])[0]
        self.phi_left = phim1                               # phi_a(t_{n-1}^+)
        # K_ab = int phi_b'(t) phi_a(t) dt = int dphi_b/dthat phi_a dthat
        self.K = np.einsum("q,qa,qb->ab", wg, phi, dphi) + np.outer(phim1, phim1)
        self.M = 0.5 * tau * np.einsum("q,qa,qb->ab", wg, phi, phi)
        self.w = 0.5 * tau * self.omega                     # diagonal of M
        self.C = phim1.copy()

    def times(self, t0):
        """Radau time points t_n^a of the slab (t0, t0 + tau]."""
        return t0 + 0.5 * self.tau * (self.that + 1.0)

    def eval_basis(self, that):
        """phi_a(that) for arbitrary reference times (used by transfers and the midpoint)."""
        if self.k == 0:
            return np.ones((len(np.atleast_1d(that)), 1))
        return lagrange_eval(self.that, that)


# ----------------------------------------------------------------------------- space
class SpaceRef:
    """Reference-cell data for Q_{r+1}^d / P_r^disc with n_q Gauss points per direction."""

    def __init__(self, d, r, nq=None):
        self.d, self.r = d, r
        self.n = r + 2                                  # velocity nodes per direction
        self.nq = nq if nq is not None else r + 2       # quadrature points per direction
        self.nodes = gauss_lobatto_01(self.n)
        self.qx, self.qw = gauss_legendre_01(self.nq)
        self.modes = pressure_modes(r, d)
        self.np = len(self.modes)
        # 1D tables at quadrature points
        self.B1 = lagrange_eval(self.nodes, self.qx)       # [nq, n]
        self.D1 = lagrange_deriv(self.nodes, self.qx)      # [nq, n]
        self.P1 = legendre01(r, self.qx)                   # [nq, r+1]
        self.dP1 = legendre01_deriv(r, self.qx)
        # full tensor tables (x fastest) at volume quadrature points
        self.qpts = np.array(list(itertools.product(*([self.qx] * d))))[:, ::-1]  # [Q, d] x fastest
        self.qwts = np.prod(np.array(list(itertools.product(*([self.qw] * d)))), axis=1)
        self.phi, self.dphi = self.velocity_basis(self.qpts)
        self.psi = self.pressure_basis(self.qpts)

    def local_node_multi(self):
        """Multi-index (ix, iy[, iz]) of each local velocity node, x fastest."""
        return np.array(list(itertools.product(*([range(self.n)] * self.d))))[:, ::-1]

    def velocity_basis(self, pts):
        """phi[p, i] and reference gradients dphi[p, i, l] of the tensor Lagrange basis."""
        pts = np.atleast_2d(pts)
        d, n = self.d, self.n
        Lv = [lagrange_eval(self.nodes, pts[:, l]) for l in range(d)]
        Ld = [lagrange_deriv(self.nodes, pts[:, l]) for l in range(d)]
        idx = self.local_node_multi()
        phi = np.ones((len(pts), len(idx)))
        dphi = np.ones((len(pts), len(idx), d))
        for i, mi in enumerate(idx):
            for l in range(d):
                phi[:, i] *= Lv[l][:, mi[l]]
                for g in range(d):
                    dphi[:, i, g] *= (Ld[l][:, mi[l]] if g == l else Lv[l][:, mi[l]])
        return phi, dphi

    def pressure_basis(self, pts):
        """psi[p, m] = prod_l P_{m_l}(2 x_l - 1) on the reference cell (mapped P_r^disc)."""
        pts = np.atleast_2d(pts)
        Lg = [legendre01(self.r, pts[:, l]) for l in range(self.d)]
        psi = np.ones((len(pts), self.np))
        for m, mi in enumerate(self.modes):
            for l in range(self.d):
                psi[:, m] *= Lg[l][:, mi[l]]
        return psi

    def face_points(self, axis, side):
        """Reference points and weights of the face x_axis = side (Gauss rule on the face)."""
        d = self.d
        others = [l for l in range(d) if l != axis]
        grid = list(itertools.product(*([range(self.nq)] * (d - 1))))
        pts = np.zeros((len(grid), d))
        wts = np.ones(len(grid))
        for g, gi in enumerate(grid):
            gi = gi[::-1]                                  # first tangential coordinate fastest
            for t, l in enumerate(others):
                pts[g, l] = self.qx[gi[t]]
                wts[g] *= self.qw[gi[t]]
            pts[g, axis] = float(side)
        return pts, wts
