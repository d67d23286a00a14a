"""Pins of the oracle's residual and Jacobian (no GPU).

* brute force: the spatial operator on a 2x2 Cartesian mesh evaluated from the bilinear
  forms (Eq. ns-form-tp, def-b-gam, Defcp, bttp) with global basis functions built
  independently (scipy Lagrange polynomials, point location, 10-point Gauss per cell/face);
* J = derivative of R (central differences, error O(eps^2));
* the constant pressure of every time node is in the null space of J (pure Dirichlet);
* polynomial solutions in the discrete space are reproduced exactly (consistency of every
  term, including the Nitsche and boundary convection terms, and of DG in time);
* the manufactured convergence test reproduces the errors printed in the paper's
  Table conv-ns (tests/golden/conv_ns_table.txt).
"""
import os

import numpy as np
import pytest
import warnings

from scipy.interpolate import lagrange
from scipy.special import eval_legendre

from oracle import forms, marching, problems
from oracle.mesh import Mesh, Space, uniform_vertices
from oracle.reference import TimeData

HERE = os.path.dirname(os.path.abspath(__file__))


def perturbed_vertices(d, n, amp, seed):
    rng = np.random.default_rng(seed)
    V = uniform_vertices(d, n)
    inner = np.all((V > 1e-12) & (V < 1 - 1e-12), axis=1)
    V[inner] += amp / n * rng.uniform(-1, 1, (inner.sum(), d))
    return V


# ----------------------------------------------------------------------------- brute force
def _brute_force_operator(n, r, nu, V, g1, g2, with_mass=False):
    """Spatial Jacobian [[A, B^T], [B, 0]] of one time node on the Cartesian n x n mesh (and,
    with_mass, the velocity mass matrix of both components)."""
    gll = {3: [0.0, 0.5, 1.0], 4: [0.0, 0.5 - 5 ** 0.5 / 10, 0.5 + 5 ** 0.5 / 10, 1.0]}[r + 2]
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", DeprecationWarning)
        polys = [lagrange(gll, np.eye(r + 2)[i]) for i in range(r + 2)]
    dpolys = [np.polyder(p) for p in polys]
    N1 = (r + 1) * n + 1
    h = 1.0 / n
    xg, wg = np.polynomial.legendre.leggauss(10)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    modes = [(s - j, j) for s in range(r + 1) for j in range(s + 1)]
    npc = len(modes)

    def basis_at(px, py):
        """All global scalar velocity basis values/gradients and pressure basis at points."""
        P = len(px)
        cx = np.minimum((px / h).astype(int), n - 1)
        cy = np.minimum((py / h).astype(int), n - 1)
        xi, eta = px / h - cx, py / h - cy
        Phi = np.zeros((P, N1 * N1))
        dPhi = np.zeros((P, N1 * N1, 2))
        Psi = np.zeros((P, n * n * npc))
        for p in range(P):
            for iy in range(r + 2):
                for ix in range(r + 2):
                    gidx = (cx[p] * (r + 1) + ix) + N1 * (cy[p] * (r + 1) + iy)
                    lx, ly = polys[ix](xi[p]), polys[iy](eta[p])
                    Phi[p, gidx] = lx * ly
                    dPhi[p, gidx, 0] = dpolys[ix](xi[p]) / h * ly
                    dPhi[p, gidx, 1] = lx * dpolys[iy](eta[p]) / h
            c = cx[p] + n * cy[p]
            for m, (i, j) in enumerate(modes):
                Psi[p, c * npc + m] = eval_legendre(i, 2 * xi[p] - 1) * eval_legendre(j, 2 * eta[p] - 1)
        return Phi, dPhi, Psi

    nn = N1 * N1
    Nv, Np = 2 * nn, n * n * npc
    A = np.zeros((Nv, Nv))
    B = np.zeros((Np, Nv))
    # volume
    px, py, pw = [], [], []
    for cy in range(n):
        for cx in range(n):
            for a in range(10):
                for b in range(10):
                    px.append((cx + xg[a]) * h); py.append((cy + xg[b]) * h); pw.append(wg[a] * wg[b] * h * h)
    px, py, pw = map(np.array, (px, py, pw))
    Phi, dPhi, Psi = basis_at(px, py)
    Ms = np.einsum("p,pi,pj->ij", pw, Phi, Phi)
    v = np.stack([Phi @ V[:nn], Phi @ V[nn:]], -1)
    for c in range(2):
        for e in range(2):
            blk = np.zeros((nn, nn))
            if c == e:
                blk += nu * np.einsum("p,pil,pjl->ij", pw, dPhi, dPhi)
                blk -= np.einsum("p,pj,pl,pil->ij", pw, Phi, v, dPhi)
            blk -= np.einsum("p,p,pj,pi->ij", pw, v[:, c], Phi, dPhi[:, :, e])
            A[c * nn:(c + 1) * nn, e * nn:(e + 1) * nn] += blk
        B[:, c * nn:(c + 1) * nn] -= np.einsum("p,pm,pj->mj", pw, Psi, dPhi[:, :, c])
    # faces
    hn = h / ((r + 1) * (r + 2))
    for axis in range(2):
        for side in (0, 1):
            nrm = np.zeros(2); nrm[axis] = 1.0 if side else -1.0
            px, py, pw = [], [], []
            for cell in range(n):
                for a in range(10):
                    t = (cell + xg[a]) * h
                    fixed = 1.0 - 1e-14 if side else 1e-14
                    if axis == 0:
                        px.append(fixed); py.append(t)
                    else:
                        px.append(t); py.append(fixed)
                    pw.append(wg[a] * h)
            px, py, pw = map(np.array, (px, py, pw))
            Phi, dPhi, Psi = basis_at(px, py)
            v = np.stack([Phi @ V[:nn], Phi @ V[nn:]], -1)
            y = v @ nrm
            dn = dPhi @ nrm
            ypm = 0.5 * (np.abs(y) + y) - (np.abs(y) - y)
            for c in range(2):
                for e in range(2):
                    blk = np.zeros((nn, nn))
                    if c == e:
                        blk += -nu * np.einsum("p,pj,pi->ij", pw, dn, Phi)
                        blk += -nu * np.einsum("p,pj,pi->ij", pw, Phi, dn)
                        blk += nu * g1 / hn * np.einsum("p,pj,pi->ij", pw, Phi, Phi)
                        blk += np.einsum("p,p,pj,pi->ij", pw, ypm, Phi, Phi)
                    blk += g2 / hn * nrm[c] * nrm[e] * np.einsum("p,pj,pi->ij", pw, Phi, Phi)
                    blk += nrm[e] * np.einsum("p,p,p,pj,pi->ij", pw, 0.5 * (3 - np.sign(y)), v[:, c], Phi, Phi)
                    A[c * nn:(c + 1) * nn, e * nn:(e + 1) * nn] += blk
                B[:, c * nn:(c + 1) * nn] += nrm[c] * np.einsum("p,pm,pj->mj", pw, Psi, Phi)
    if with_mass:
        return A, B, np.kron(np.eye(2), Ms)
    return A, B


@pytest.mark.parametrize("n,r", [(1, 1), (2, 1), (2, 2)])
@pytest.mark.parametrize("state", ["zero", "affine"])
def test_brute_force_spatial_operator(n, r, state):
    """The state is zero or affine with a fixed sign of v.n on every boundary face, so that the
    (r+2)-point Gauss rule integrates every term exactly and the brute force may use any rule."""
    s = Space(Mesh(2, n, uniform_vertices(2, n)), r)
    nu, tau = 0.03, 0.2
    td = TimeData(0, tau)
    lay = forms.SlabLayout(s, 0)
    U = np.zeros(lay.Nst)
    if state == "affine":
        U[:s.Nv] = forms.interpolate_velocity(s, lambda x: np.stack(
            [1.0 + 0.5 * x[:, 0] + 0.3 * x[:, 1], -1.0 + 0.4 * x[:, 0] + 0.2 * x[:, 1]], -1))
    J = forms.jacobian(s, td, U, nu).toarray()
    M = forms.mass_velocity(s).toarray()
    A_or = (J[:s.Nv, :s.Nv] - M) / tau
    B_or = J[s.Nv:, :s.Nv] / tau
    A_bf, B_bf = _brute_force_operator(n, r, nu, U[:s.Nv], 10.0, 10.0)
    assert np.abs(A_or - A_bf).max() < 1e-11 * np.abs(A_bf).max()
    assert np.abs(B_or - B_bf).max() < 1e-12 * np.abs(B_bf).max()
    assert np.allclose(J[:s.Nv, s.Nv:], J[s.Nv:, :s.Nv].T, atol=1e-15)   # J^21 = J^12^T
    assert np.abs(J[s.Nv:, s.Nv:]).max() == 0.0


# ----------------------------------------------------------------------------- derivative, null space
CASES = [(2, 3, 2, 2, "MMS2D"), (2, 2, 1, 1, "TG2D"), (3, 2, 1, 1, "MMS3D"), (3, 2, 2, 0, "TG3D")]


@pytest.mark.parametrize("d,n,r,k,pname", CASES)
def test_jacobian_is_derivative_of_residual(d, n, r, k, pname):
    rng = np.random.default_rng(11)
    s = Space(Mesh(d, n, perturbed_vertices(d, n, 0.2, 3)), r)
    td = TimeData(k, 0.07)
    lay = forms.SlabLayout(s, k)
    prob = problems.make(pname, 0.02)
    U = rng.uniform(-1, 1, lay.Nst)
    Vp = rng.uniform(-1, 1, lay.Nv)
    x = rng.uniform(-1, 1, lay.Nst)
    Jx = forms.jacobian(s, td, U, prob.nu) @ x
    # R is quadratic in U away from the kinks of (v.n)^+- on the boundary, so central
    # differences are exact up to roundoff; a small eps keeps every face point off its kink.
    eps = 1e-5
    fd = (forms.residual(s, td, U + eps * x, Vp, prob, 0.1)
          - forms.residual(s, td, U - eps * x, Vp, prob, 0.1)) / (2 * eps)
    assert np.abs(fd - Jx).max() < 1e-8 * np.abs(Jx).max()


@pytest.mark.parametrize("d,n,r,k", [(2, 3, 2, 2), (3, 2, 1, 1), (3, 2, 2, 1)])
def test_constant_pressure_null_space(d, n, r, k):
    rng = np.random.default_rng(2)
    s = Space(Mesh(d, n, perturbed_vertices(d, n, 0.25, 4)), r)
    td = TimeData(k, 0.1)
    lay = forms.SlabLayout(s, k)
    U = rng.uniform(-1, 1, lay.Nst)
    J = forms.jacobian(s, td, U, 0.01)
    scale = abs(J).max()
    for a in range(k + 1):
        z = np.zeros(lay.Nst)
        z[lay.poff(a) + np.arange(s.mesh.ncells) * s.npc] = 1.0      # mode 0 = constant
        assert np.abs(J @ z).max() < 1e-14 * scale * s.mesh.ncells
        assert np.abs(J.T @ z).max() < 1e-14 * scale * s.mesh.ncells


# ----------------------------------------------------------------------------- exactness
class _PolyFlow(problems.Problem):
    """v = (a + b t)(y^2, x^2), p = (a + b t)(x + y - 1): div-free, in Q_2 x P_1, linear in t."""

    def __init__(self, nu, a, b):
        super().__init__(nu)
        self.a, self.b = a, b

    def v(self, x, t):
        s = self.a + self.b * t
        return s * np.stack([x[..., 1] ** 2, x[..., 0] ** 2], -1)

    def g(self, x, t):
        return self.v(x, t)

    def v0(self, x):
        return self.v(x, 0.0)

    def f(self, x, t):
        X, Y = x[..., 0], x[..., 1]
        s = self.a + self.b * t
        return np.stack([self.b * Y * Y + s * s * 2 * X * X * Y - 2 * self.nu * s + s,
                         self.b * X * X + s * s * 2 * X * Y * Y - 2 * self.nu * s + s], -1)


@pytest.mark.parametrize("r,k,a,b,t0", [(1, 0, 1.0, 0.0, 0.0), (1, 1, 1.0, 0.0, 0.5),
                                        (1, 2, 0.0, 1.0, 0.3), (2, 2, 0.5, 1.0, 0.3)])
def test_polynomial_solution_is_reproduced(r, k, a, b, t0):
    prob = _PolyFlow(0.1, a, b)
    s = Space(Mesh(2, 2, uniform_vertices(2, 2)), r)
    td = TimeData(k, 0.1)
    lay = forms.SlabLayout(s, k)
    Vprev = forms.interpolate_velocity(s, lambda x: prob.v(x, t0))
    U, _ = marching.newton_direct(s, td, np.zeros(lay.Nst), Vprev, prob, t0, tol=1e-14)
    for i, t in enumerate(td.times(t0)):
        Vex = forms.interpolate_velocity(s, lambda x: prob.v(x, t))
        assert np.abs(lay.v(U, i) - Vex).max() < 1e-10
        pq = forms.pressure_at(s, lay.p(U, i), s.ref.psi)
        assert np.abs(pq - (a + b * t) * (s.xq[..., 0] + s.xq[..., 1] - 1)).max() < 1e-10


# ----------------------------------------------------------------------------- convergence
def _golden():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "conv_ns_table.txt")):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows[(int(f[0]), int(f[1]))] = [float(x) for x in f[2:]]
    return rows


@pytest.mark.slow
@pytest.mark.parametrize("r,ninv", [(3, 2), (3, 4), (4, 2)])
def test_manufactured_convergence_matches_paper_table(r, ninv):
    prob = problems.make("MMS2D", 1e-2)
    s = Space(Mesh(2, ninv, uniform_vertices(2, ninv)), r)
    td, sols = marching.march(s, r, 1.0 / ninv, ninv, prob)
    ev, ep, eh, ed = marching.spacetime_errors(s, td, sols, prob)
    ref = _golden()[(r, ninv)]
    for got, want in zip((ev, ep, eh, ed), ref):
        assert abs(got - want) / want < 0.03, (got, want)
