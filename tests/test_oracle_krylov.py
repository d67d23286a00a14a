"""Pins of the oracle's outer solvers (Sec. 4.1, Alg. 1-2) against facts independent of it:

* FGMRES solves a nonsymmetric system to the requested tolerance (checked by the true residual
  and numpy's dense solve), with and without restarts, takes one step with the exact inverse as
  preconditioner, and stays correct with a preconditioner that changes every call (the flexible
  property: the update is built from the preconditioned vectors actually used);
* the backtracking interpolation returns the exact minimiser of a quadratic (one failed step)
  and of a cubic (two failed steps) merit function -- the closed forms of the safeguarded
  quadratic / cubic line search;
* Newton (Alg. 1 with Alg. 2) reaches the root of a small nonlinear algebraic system that scipy
  finds independently, with its residual history decreasing to the tolerance;
* a full slab solve with the multigrid preconditioner equals the slab solution of Newton with
  sparse direct linear solves.
"""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import forms, krylov, marching, problems
from paper_2602_13841_gb300 import inputs


def _system(n=40, seed=0):
    rng = np.random.default_rng(seed)
    A = 4.0 * np.eye(n) + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    return A, b


@pytest.mark.parametrize("restart,maxit", [(40, 40), (8, 200)])
def test_fgmres_solves_to_tolerance(restart, maxit):
    A, b = _system()
    x, its, ratios = krylov.fgmres(lambda v: A @ v, b, lambda v: v, 1e-11, restart, maxit)
    assert np.linalg.norm(b - A @ x) <= 1.01e-11 * np.linalg.norm(b)
    assert np.abs(x - np.linalg.solve(A, b)).max() < 1e-9 * np.abs(x).max()
    assert its == len(ratios) <= maxit


def test_fgmres_exact_preconditioner_takes_one_step():
    A, b = _system(seed=1)
    Ainv = np.linalg.inv(A)
    x, its, _ = krylov.fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, 1e-10, 30, 30)
    assert its == 1
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)


def test_fgmres_is_flexible():
    """A different approximate inverse at every call (inverse of A plus a call-dependent
    perturbation): the returned x still meets the tolerance in the true residual."""
    A, b = _system(seed=2)
    rng = np.random.default_rng(5)
    calls = [0]

    def M(v):
        calls[0] += 1
        E = 0.3 * rng.standard_normal(A.shape) / np.sqrt(A.shape[0])
        return np.linalg.solve(A + E, v)
    x, its, _ = krylov.fgmres(lambda v: A @ v, b, M, 1e-10, 40, 40)
    assert calls[0] >= its > 1
    assert np.linalg.norm(b - A @ x) <= 1.01e-10 * np.linalg.norm(b)


def test_line_search_interpolation_is_exact_on_quadratic_and_cubic():
    phi0, g0 = 2.0, -3.0
    c2 = 1.7                       # phi(a) = phi0 + g0 a + c2 a^2, minimiser -g0 / (2 c2)
    q = lambda a: phi0 + g0 * a + c2 * a * a
    a = krylov._interp_step(1.0, q(1.0), None, None, phi0, g0)
    assert abs(a - (-g0 / (2 * c2))) < 1e-14
    ca, cb = 0.8, 1.1              # phi(a) = phi0 + g0 a + cb a^2 + ca a^3
    cu = lambda a: phi0 + g0 * a + cb * a * a + ca * a ** 3
    a = krylov._interp_step(0.6, cu(0.6), 1.0, cu(1.0), phi0, g0)
    amin = (-cb + np.sqrt(cb * cb - 3 * ca * g0)) / (3 * ca)
    assert abs(a - amin) < 1e-12
    assert abs(g0 + 2 * cb * amin + 3 * ca * amin * amin) < 1e-12


class _ExactPre:
    """mg stand-in: setup(U) stores J(U); vcycle solves with it exactly."""

    def __init__(self, jac):
        self.jac, self.J = jac, None

    def setup(self, U):
        self.J = self.jac(U)

    def vcycle(self, r):
        return np.linalg.solve(self.J, r)


def test_newton_finds_the_root_of_an_algebraic_system():
    n = 12
    rng = np.random.default_rng(3)
    A = 3.0 * np.eye(n) + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n) * 3.0
    R = lambda U: A @ U + U ** 3 - b
    Jm = lambda U: A + np.diag(3.0 * U ** 2)
    root = so.fsolve(R, np.zeros(n), fprime=Jm, xtol=1e-13)
    prm = dict(krylov.DEFAULTS)
    prm.update(rtol=1e-12, atol=0.0, project=lambda U: U)
    mg = _ExactPre(Jm)
    X, st = krylov.newton_slab(np.zeros(n), None, 0.0, R, lambda U, x: Jm(U) @ x,
                               lambda z: float(np.linalg.norm(z)), lambda a, c: float(a @ c), mg, prm)
    assert st.res <= 1e-12 * st.res0
    assert np.abs(X - root).max() < 1e-10 * np.abs(root).max()
    res = [h[0] for h in st.history]
    assert res[-1] < res[0] and 1 <= st.newton_its <= prm["maxit"]


def test_slab_solve_equals_direct_newton():
    d, n, r, k, nu, tau = 2, 4, 1, 1, 1e-2, 0.1
    prob = problems.make("TG2D", nu)
    verts = inputs.vertices(d, n, 0.1, 8)
    S = krylov.SlabSolver(d, n, r, k, verts, tau, prob, rtol=1e-11, atol=0.0)
    L = S.L
    Vp = forms.interpolate_velocity(L.space, prob.v0)
    U0 = np.concatenate([np.tile(Vp, k + 1), np.zeros((k + 1) * L.lay.Np)])
    X, st = S.solve(U0, Vp, 0.0)
    Ud, _ = marching.newton_direct(L.space, L.td, U0, Vp, prob, 0.0, tol=1e-14)
    nv = (k + 1) * L.lay.Nv
    assert st.res <= 1e-11 * st.res0
    assert np.abs(X[:nv] - Ud[:nv]).max() < 1e-8 * np.abs(Ud[:nv]).max()
    assert np.abs(X[nv:] - Ud[nv:]).max() < 1e-7 * max(np.abs(Ud[nv:]).max(), 1.0)
