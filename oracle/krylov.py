"""FGMRES and the inexact Newton-Krylov method (oracle; test infrastructure).

* FGMRES (Saad 1993): right-preconditioned flexible GMRES, one V-cycle per iteration,
  modified Gram-Schmidt, Givens rotations, restart m, iteration cap; stops when the
  Euclidean residual estimate |g_{j+1}| <= eta ||b|| (Sec. 4.1-4.2; the paper gives no inner
  product for FGMRES, the Euclidean one is used).
* Newton (Alg. 1): Eisenstat-Walker forcing eta = clamp(c_eta eta (||r||/||r_prev||)^theta),
  smoother rebuild triggers (rho_prev >= theta_N, kappa_prev >= max(theta_L kappa_ref,
  kappa_abs), FGMRES stagnation over s iterations with ratio >= vartheta), mass-weighted norm
  ||.||_M (Sec. 4.1), pressure mean removed after every step.
* Armijo (Alg. 2) on phi(alpha) = 1/2 ||R(X + alpha dX)||_M^2 with g0 = r^T M J dX (the
  derivative of phi at 0), nonmonotone window of the last M accepted merits kept across the
  Newton steps of one slab, safeguarded quadratic (one failure) / cubic (two failures)
  interpolation clamped to [0.1 alpha, 0.5 alpha], at most ls_maxbt backtracks, alpha_min
  returned when no step is accepted.
"""
import numpy as np

from . import forms
from .multigrid import Multigrid


def fgmres(A, b, M, tol, restart=30, maxit=50, x0=None):
    """Solve A x = b with right preconditioner M (callables). Returns x, iterations, ratios."""
    n = len(b)
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    its = 0
    ratios = []
    if bnorm == 0.0:
        return x, 0, ratios
    while its < maxit:
        r = b - A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        m = min(restart, maxit - its)
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = M(V[j])
            w = A(Z[j])
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            prev = abs(g[j])
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            ratios.append(abs(g[j + 1]) / max(prev, 1e-300))
            if abs(g[j + 1]) <= tol * bnorm:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Z[:j_done].T @ y
        if abs(g[j_done]) <= tol * bnorm:
            break
    return x, its, ratios


class NewtonStats:
    def __init__(self):
        self.newton_its = 0
        self.gmres_its = 0
        self.rebuilds = 0
        self.backtracks = 0
        self.res0 = self.res = 0.0
        self.history = []


def _interp_step(a1, f1, a2, f2, phi0, g0):
    """Safeguarded backtracking step (Dennis & Schnabel, Alg. A6.3.1)."""
    if a2 is None:
        den = 2.0 * (f1 - phi0 - g0 * a1)
        return None if den <= 0 else -g0 * a1 * a1 / den
    r1 = f1 - phi0 - g0 * a1
    r2 = f2 - phi0 - g0 * a2
    dd = a1 - a2
    a = (r1 / a1 ** 2 - r2 / a2 ** 2) / dd
    b = (-a2 * r1 / a1 ** 2 + a1 * r2 / a2 ** 2) / dd
    if a == 0.0:
        return None if b == 0 else -g0 / (2.0 * b)
    disc = b * b - 3.0 * a * g0
    if disc < 0:
        return None
    return (-b + np.sqrt(disc)) / (3.0 * a)


def newton_slab(U0, Vprev, t0, residual, jac_apply, mnorm, mdot, mg, prm, stats=None):
    """Alg. 1 for one slab.  residual(U) -> R; jac_apply(U, x) -> J(U) x; mnorm/mdot: the
    M-weighted norm and inner product; mg: object with setup(U) and vcycle(r)."""
    st = stats or NewtonStats()
    eps = 1e-30
    X = U0.copy()
    r = residual(X)
    n0 = mnorm(r)
    st.res0 = n0
    nprev, eta, rho_prev, kap_prev, kap_ref = n0, prm["ew_eta0"], 1.0, 1, 1
    window = [0.5 * n0 * n0]
    k = 0
    while mnorm(r) > max(prm["atol"], prm["rtol"] * n0) and k < prm["maxit"]:
        nr = mnorm(r)
        if rho_prev >= prm["thetaN"] or kap_prev >= max(prm["thetaL"] * kap_ref, prm["kappa_abs"]):
            mg.setup(X)
            st.rebuilds += 1
            kap_ref = max(1, kap_prev)
        if k > 0:
            eta = min(max(prm["ew_c"] * eta * (nr / max(nprev, eps)) ** prm["ew_theta"], prm["ew_min"]),
                      prm["ew_max"])
        dX, kap, ratios = fgmres(lambda v: jac_apply(X, v), -r, mg.vcycle, eta,
                                 prm["restart"], prm["gmres_maxit"])
        st.gmres_its += kap
        # Armijo (Alg. 2)
        alpha = prm["ls_lambda0"]
        phi0 = 0.5 * nr * nr
        g0 = mdot(r, jac_apply(X, dX))
        fails = []
        accepted = False
        for bt in range(prm["ls_maxbt"] + 1):
            if alpha <= prm["ls_alpha_min"]:
                break
            rt = residual(X + alpha * dX)
            phit = 0.5 * mnorm(rt) ** 2
            phimax = max(window) if prm["ls_window"] > 0 else phi0
            if phit <= phimax + prm["ls_c"] * alpha * g0:
                accepted = True
                break
            fails.insert(0, (alpha, phit))
            a2, f2 = fails[1] if len(fails) > 1 else (None, None)
            ai = _interp_step(fails[0][0], fails[0][1], a2, f2, phi0, g0)
            st.backtracks += 1
            alpha = alpha * prm["ls_tau"] if ai is None else min(max(ai, 0.1 * alpha), 0.5 * alpha)
        if not accepted:
            alpha = max(alpha, prm["ls_alpha_min"])
            rt = residual(X + alpha * dX)
            phit = 0.5 * mnorm(rt) ** 2
        window.append(phit)
        window = window[-max(prm["ls_window"], 1):]
        X = X + alpha * dX
        X = prm["project"](X)
        nprev = nr
        r = residual(X)
        rho_prev = mnorm(r) / max(nprev, eps)
        kap_prev = max(1, kap)
        st.history.append((mnorm(r), kap, alpha))
        s = prm["stag_s"]
        if len(ratios) >= s and all(q >= prm["stag_theta"] for q in ratios[-s:]):
            mg.setup(X)
            st.rebuilds += 1
        k += 1
    st.newton_its = k
    st.res = mnorm(r)
    return X, st


DEFAULTS = dict(rtol=1e-8, atol=1e-12, maxit=20, ew_eta0=0.4, ew_c=0.5, ew_theta=1.5, ew_min=1e-3,
                ew_max=0.8, ls_lambda0=1.0, ls_c=1e-4, ls_tau=0.5, ls_alpha_min=1e-3, ls_maxbt=5,
                ls_window=5, restart=50, gmres_maxit=50, thetaN=1.0, thetaL=2.0, kappa_abs=50,
                stag_s=3, stag_theta=0.95)


class SlabSolver:
    """Newton-FGMRES with hp-STMG on one configuration (all FP64)."""

    def __init__(self, d, n, r, k, vertices, tau, prob, omega=None, max_h=-1, omega_p=1.0, nu1=1, nu2=1,
                 keep_k=False, smoother="vanka", nu_tc=0, **overrides):
        self.mg = Multigrid(d, n, r, k, vertices, tau, prob.nu, omega=omega, max_h=max_h, omega_p=omega_p,
                            nu1=nu1, nu2=nu2, keep_k=keep_k, smoother=smoother, nu_tc=nu_tc)
        self.L = self.mg.levels[0]
        self.prob = prob
        self.M = forms.slab_mass(self.L.space, self.L.td)
        self.prm = dict(DEFAULTS)
        self.prm.update(overrides)
        s = self.L.space
        self.pw = np.einsum("kq,qm->km", s.JxW, s.ref.psi).ravel()
        self.vol = s.JxW.sum()
        self.prm["project"] = self.project

    def project(self, U):
        """Remove the pressure mean at every time node (L^2_0 representative)."""
        lay = self.L.lay
        U = U.copy()
        for a in range(self.L.k + 1):
            P = U[lay.poff(a):lay.poff(a) + lay.Np]
            mean = np.dot(self.pw, P) / self.vol
            P[np.arange(0, lay.Np, self.L.space.npc)] -= mean
        return U

    def solve(self, U0, Vprev, t0):
        L = self.L
        res = lambda U: forms.residual(L.space, L.td, U, Vprev, self.prob, t0)
        jac = lambda U, x: forms.jacobian(L.space, L.td, U, self.prob.nu) @ x
        mnorm = lambda Z: float(np.sqrt(max(Z @ (self.M @ Z), 0.0)))
        mdot = lambda a, b: float(a @ (self.M @ b))
        return newton_slab(U0, Vprev, t0, res, jac, mnorm, mdot, self.mg, self.prm)
