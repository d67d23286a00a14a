"""Pins of the oracle's Vanka smoother (Sec. 4.3, Eq. LVS, vanka0, DefTildeHn, DefVnAst) against
objects built without the oracle:

* one additive sweep equals the dense formula d + W sum_K R_K^T (R_K J~ R_K^T)^{-1} R_K (b - J d),
  with J and the midpoint surrogate J~ assembled from the brute-force spatial operator (scipy
  Lagrange basis, 10-point Gauss rule), the textbook DG(1) time matrices (Radau nodes -1/3, 1:
  K = [[9/8, 3/8], [-9/8, 5/8]], M = tau/2 diag(3/2, 1/2)), patch index lists written out from
  the mesh numbering, and the surrogate state v* = the analytic field at the slab midpoint.  A
  patch taken from the element matrices instead of the global submatrix, a dropped pressure
  relaxation weight, another evaluation time t*, or a non-additive sweep each fails it;
* the midpoint state: for a velocity polynomial in time, midpoint_velocity equals the field at
  t_{n-1} + tau / 2 (closed-form Radau nodes of DG(1) and DG(2)).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import multigrid
from oracle.mesh import uniform_vertices
from tests.test_oracle_forms import _brute_force_operator


def _affine(x, y, c):
    return np.stack([c[0] + c[1] * x + c[2] * y, c[3] + c[4] * x + c[5] * y], -1)


# v = F0 + that * F1 (that: reference time in [-1, 1]); v.n keeps one sign on every boundary face
F0 = (1.0, 0.5, 0.3, -1.0, 0.4, 0.2)
F1 = (0.15, -0.06, 0.03, 0.12, 0.03, -0.09)


def _nodes_xy(n, r):
    """Coordinates of the global velocity nodes (x fastest) from the closed-form GLL points."""
    g = {3: [0.0, 0.5, 1.0], 4: [0.0, 0.5 - 5 ** 0.5 / 10, 0.5 + 5 ** 0.5 / 10, 1.0]}[r + 2]
    x1 = np.array([(c + g[i]) / n for c in range(n) for i in range(r + 1)] + [1.0])
    X, Y = np.meshgrid(x1, x1)          # rows: y, columns: x
    return X.ravel(), Y.ravel()


def _patch_lists(n, r, k):
    """Global slab indices of every cell patch: both velocity components at every node of the
    cell and every pressure mode of the cell, at every time node."""
    N1 = (r + 1) * n + 1
    nn = N1 * N1
    npc = (r + 1) * (r + 2) // 2
    Nv, Np = 2 * nn, n * n * npc
    out = []
    for cy in range(n):
        for cx in range(n):
            nodes = [(cx * (r + 1) + ix) + N1 * (cy * (r + 1) + iy) for iy in range(r + 2) for ix in range(r + 2)]
            cell = cx + n * cy
            idx = []
            for a in range(k + 1):
                for c in range(2):
                    idx += [a * Nv + c * nn + j for j in nodes]
            for a in range(k + 1):
                idx += [(k + 1) * Nv + a * Np + cell * npc + m for m in range(npc)]
            out.append(np.array(idx))
    return out


def _slab_matrix(K, w, Ms, As, B):
    """[[K (x) M + blockdiag_a(w_a A_a), blockdiag_a(w_a B^T)], [blockdiag_a(w_a B), 0]]."""
    kp1 = len(w)
    Nv, Np = Ms.shape[0], B.shape[0]
    J = np.zeros((kp1 * (Nv + Np),) * 2)
    for a in range(kp1):
        for b in range(kp1):
            J[a * Nv:(a + 1) * Nv, b * Nv:(b + 1) * Nv] = K[a][b] * Ms
        J[a * Nv:(a + 1) * Nv, a * Nv:(a + 1) * Nv] += w[a] * As[a]
        po = kp1 * Nv + a * Np
        J[a * Nv:(a + 1) * Nv, po:po + Np] = w[a] * B.T
        J[po:po + Np, a * Nv:(a + 1) * Nv] = w[a] * B
    return J


@pytest.mark.parametrize("n,r", [(2, 1), (3, 1), (2, 2)])
def test_vanka_sweep_equals_the_dense_patch_formula(n, r):
    k, nu, tau, omega, omega_p = 1, 0.03, 0.2, 0.3, 1.0
    that = np.array([-1.0 / 3.0, 1.0])
    K = [[9 / 8, 3 / 8], [-9 / 8, 5 / 8]]
    w = 0.5 * tau * np.array([1.5, 0.5])
    X, Y = _nodes_xy(n, r)
    f0, f1 = _affine(X, Y, F0), _affine(X, Y, F1)
    Va = [np.concatenate([(f0 + t * f1)[:, 0], (f0 + t * f1)[:, 1]]) for t in that]
    vstar = np.concatenate([f0[:, 0], f0[:, 1]])          # the field at reference time 0
    # boundary normal velocities keep their sign (the boundary convection has no kink there)
    for V in Va + [vstar]:
        nn = len(X)
        vx, vy = V[:nn], V[nn:]
        bnd_x = (X < 1e-12) | (X > 1 - 1e-12)
        bnd_y = (Y < 1e-12) | (Y > 1 - 1e-12)
        assert np.abs(vx[bnd_x]).min() > 0.2 and np.abs(vy[bnd_y]).min() > 0.2
    A0, B, Ms = _brute_force_operator(n, r, nu, Va[0], 10.0, 10.0, with_mass=True)
    A1, _ = _brute_force_operator(n, r, nu, Va[1], 10.0, 10.0)
    As, _ = _brute_force_operator(n, r, nu, vstar, 10.0, 10.0)
    J = _slab_matrix(K, w, Ms, [A0, A1], B)
    Jt = _slab_matrix(K, w, Ms, [As, As], B)
    N = J.shape[0]
    kp1Nv = 2 * Ms.shape[0]
    Wt = np.where(np.arange(N) < kp1Nv, omega, omega_p)
    rng = np.random.default_rng(5)
    b = rng.uniform(-1, 1, N)
    d = rng.uniform(-1, 1, N)
    res = b - J @ d
    upd = np.zeros(N)
    for idx in _patch_lists(n, r, k):
        upd[idx] += np.linalg.solve(Jt[np.ix_(idx, idx)], res[idx])
    want = d + Wt * upd
    # the oracle's sweep, with its own patch matrices and midpoint state
    lvl = multigrid.Level(2, n, r, k, uniform_vertices(2, n), tau, nu)
    U = np.zeros(lvl.Nst)
    U[:kp1Nv] = np.concatenate(Va)
    sm = multigrid.Vanka(lvl, U, omega, omega_p)
    got = sm.sweep(sp.csr_matrix(J), b, d)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    # and the patches really are global submatrices: the element-local variant differs
    assert np.abs(got - d).max() > 1e-3


@pytest.mark.parametrize("k", [1, 2])
def test_midpoint_state_is_the_field_at_the_slab_midpoint(k):
    nodes = {1: [-1.0 / 3.0, 1.0], 2: [(-1 - 6 ** 0.5) / 5, (-1 + 6 ** 0.5) / 5, 1.0]}[k]
    n, r = 2, 1
    lvl = multigrid.Level(2, n, r, k, uniform_vertices(2, n), 0.3, 0.01)
    rng = np.random.default_rng(7)
    Nv = lvl.lay.Nv
    coef = rng.uniform(-1, 1, (k + 1, Nv))             # V(that) = sum_j coef_j that^j, degree k
    U = np.zeros(lvl.Nst)
    for a, t in enumerate(nodes):
        U[a * Nv:(a + 1) * Nv] = sum(coef[j] * t ** j for j in range(k + 1))
    got = multigrid.midpoint_velocity(lvl, U)
    assert np.abs(got - coef[0]).max() < 1e-13


def test_diagonal_vanka_patch_is_the_spatially_diagonal_surrogate():
    """DiagonalVanka's local solve equals the dense solve of the surrogate patch whose velocity block
    is replaced by K (x) diag(M) + W (x) diag(A) (brute-force A, M; textbook DG(1) time matrices),
    with the pressure coupling kept whole; and it differs from the full patch."""
    n, r, k, nu, tau, omega = 2, 1, 1, 0.03, 0.2, 0.3
    that = np.array([-1.0 / 3.0, 1.0])
    K = np.array([[9 / 8, 3 / 8], [-9 / 8, 5 / 8]])
    w = 0.5 * tau * np.array([1.5, 0.5])
    X, Y = _nodes_xy(n, r)
    f0, f1 = _affine(X, Y, F0), _affine(X, Y, F1)
    Va = [np.concatenate([(f0 + t * f1)[:, 0], (f0 + t * f1)[:, 1]]) for t in that]
    vstar = np.concatenate([f0[:, 0], f0[:, 1]])
    As, B, Ms = _brute_force_operator(n, r, nu, vstar, 10.0, 10.0, with_mass=True)
    Jt = _slab_matrix(K, w, Ms, [As, As], B)
    lvl = multigrid.Level(2, n, r, k, uniform_vertices(2, n), tau, nu)
    U = np.zeros(lvl.Nst)
    U[:2 * Ms.shape[0]] = np.concatenate(Va)
    dv = multigrid.DiagonalVanka(lvl, U, omega, 1.0)
    full = multigrid.Vanka(lvl, U, omega, 1.0)
    rng = np.random.default_rng(3)
    import scipy.linalg as sla
    for (idx, lu), (_, lu_full) in zip(dv.patches, full.patches):
        S = Jt[np.ix_(idx, idx)]
        nv = (k + 1) * 2 * (r + 2) ** 2                    # patch velocity DoFs
        ms_v = 2 * (r + 2) ** 2
        Sd = S.copy()
        for p in range(nv):
            for q in range(nv):
                if p % ms_v != q % ms_v:
                    Sd[p, q] = 0.0
        # the kept entries are K_ab M_ii + delta_ab w_a A_ii
        a0, i0 = 0, 3
        assert abs(Sd[i0, ms_v + i0] - K[0, 1] * Ms[idx[i0], idx[i0]]) < 1e-14 * abs(Sd).max()
        b = rng.uniform(-1, 1, len(idx))
        want = np.linalg.solve(Sd, b)
        assert np.abs(sla.lu_solve(lu, b) - want).max() < 1e-11 * np.abs(want).max()
        assert np.abs(sla.lu_solve(lu_full, b) - want).max() > 1e-6 * np.abs(want).max()


def test_exact_vanka_patches_are_submatrices_of_the_true_jacobian():
    """ExactVanka uses R_K J R_K^T with the convection at each time node's own velocity (the
    brute-force J of the first test), and differs from the surrogate when V depends on time."""
    n, r, k, nu, tau = 2, 1, 1, 0.03, 0.2
    that = np.array([-1.0 / 3.0, 1.0])
    K = [[9 / 8, 3 / 8], [-9 / 8, 5 / 8]]
    w = 0.5 * tau * np.array([1.5, 0.5])
    X, Y = _nodes_xy(n, r)
    f0, f1 = _affine(X, Y, F0), _affine(X, Y, F1)
    Va = [np.concatenate([(f0 + t * f1)[:, 0], (f0 + t * f1)[:, 1]]) for t in that]
    A0, B, Ms = _brute_force_operator(n, r, nu, Va[0], 10.0, 10.0, with_mass=True)
    A1, _ = _brute_force_operator(n, r, nu, Va[1], 10.0, 10.0)
    J = _slab_matrix(K, w, Ms, [A0, A1], B)
    lvl = multigrid.Level(2, n, r, k, uniform_vertices(2, n), tau, nu)
    U = np.zeros(lvl.Nst)
    U[:2 * Ms.shape[0]] = np.concatenate(Va)
    ex = multigrid.ExactVanka(lvl, U, 0.3, 1.0)
    sur = multigrid.Vanka(lvl, U, 0.3, 1.0)
    import scipy.linalg as sla
    rng = np.random.default_rng(9)
    for (idx, lu), (_, lus) in zip(ex.patches, sur.patches):
        b = rng.uniform(-1, 1, len(idx))
        want = np.linalg.solve(J[np.ix_(idx, idx)], b)
        assert np.abs(sla.lu_solve(lu, b) - want).max() < 1e-11 * np.abs(want).max()
        assert np.abs(sla.lu_solve(lus, b) - want).max() > 1e-8 * np.abs(want).max()
