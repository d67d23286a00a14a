"""Time marching with an exact Newton method and sparse direct solves (oracle; test infrastructure).

This is the special case of the solver of Sec. 4 in which every linear system is solved
exactly: it pins the discrete problem (Problem LocAlgNS) itself, independent of FGMRES and
multigrid.  The pressure is determined up to one constant per time node (pure Dirichlet
boundary, Remark on L^2_0); the linear systems are bordered with one mean-zero row per
time node, and the converged pressure has zero mean at every Radau node.
Space-time errors are measured with a (k+2)-point Gauss rule in time per slab and the
volume quadrature in space; the divergence error is || div v_h ||_{L2(L2)}.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from numpy.polynomial import legendre as npleg

from . import forms
from .reference import TimeData


def pressure_mean_rows(space, k):
    """[k+1, Nst] rows c_a with c_a . U = integral of the pressure at time node a."""
    lay = forms.SlabLayout(space, k)
    w = np.einsum("kq,qm->km", space.JxW, space.ref.psi).ravel()
    C = np.zeros((k + 1, lay.Nst))
    for a in range(k + 1):
        C[a, lay.poff(a):lay.poff(a) + lay.Np] = w
    return C


def bordered_solve(J, rhs, C):
    """Solve [J C^T; C 0] [x; l] = [rhs; 0] with a sparse LU."""
    nb = C.shape[0]
    Cs = sp.csr_matrix(C)
    A = sp.bmat([[J, Cs.T], [Cs, None]], format="csc")
    sol = spla.spsolve(A, np.concatenate([rhs, np.zeros(nb)]))
    return sol[:J.shape[0]]


def newton_direct(space, td, U0, Vprev, prob, t0, tol=1e-12, maxit=20, gamma=(10.0, 10.0)):
    C = pressure_mean_rows(space, td.k)
    U = U0.copy()
    r = forms.residual(space, td, U, Vprev, prob, t0, *gamma)
    r0 = np.linalg.norm(r)
    for it in range(maxit):
        if np.linalg.norm(r) <= max(tol * r0, 1e-14):
            return U, it
        J = forms.jacobian(space, td, U, prob.nu, *gamma)
        U = U - bordered_solve(J, r, C)
        r = forms.residual(space, td, U, Vprev, prob, t0, *gamma)
    return U, maxit


def march(space, k, tau, nsteps, prob, tol=1e-12):
    """March nsteps slabs from v_{0,h} (nodal interpolant of v0); returns the list of slab vectors."""
    td = TimeData(k, tau)
    lay = forms.SlabLayout(space, k)
    Vprev = forms.interpolate_velocity(space, prob.v0)
    sols = []
    for n in range(nsteps):
        U0 = np.zeros(lay.Nst)
        for a in range(k + 1):
            U0[lay.voff(a):lay.voff(a) + lay.Nv] = Vprev
        U, _ = newton_direct(space, td, U0, Vprev, prob, n * tau, tol)
        sols.append(U)
        Vprev = lay.v(U, k).copy()
    return td, sols


def spacetime_errors(space, td, sols, prob):
    """Squared-sum errors e_v L2(L2), e_p L2(L2), e_v L2(H1) seminorm, ||div v_h|| L2(L2)."""
    k, tau = td.k, td.tau
    lay = forms.SlabLayout(space, k)
    xg, wg = npleg.leggauss(k + 2)
    phi_t = td.eval_basis(xg)                     # [ng, k+1]
    ev = ep = eh = ed = 0.0
    for n, U in enumerate(sols):
        for g in range(len(xg)):
            t = n * tau + 0.5 * tau * (xg[g] + 1.0)
            wt = 0.5 * tau * wg[g]
            V = sum(phi_t[g, a] * lay.v(U, a) for a in range(k + 1))
            P = sum(phi_t[g, a] * lay.p(U, a) for a in range(k + 1))
            v, gv = forms.velocity_at_qp(space, V)
            p = forms.pressure_at(space, P, space.ref.psi)
            ve = prob.v(space.xq, t)
            pe = prob.p(space.xq, t)
            gve = _grad_exact(prob, space.xq, t)
            ev += wt * np.sum(space.JxW[..., None] * (v - ve) ** 2)
            ep += wt * np.sum(space.JxW * (p - pe) ** 2)
            eh += wt * np.sum(space.JxW[..., None, None] * (gv - gve) ** 2)
            ed += wt * np.sum(space.JxW * np.einsum("kqcc->kq", gv) ** 2)
    return np.sqrt(ev), np.sqrt(ep), np.sqrt(eh), np.sqrt(ed)


def _grad_exact(prob, x, t):
    """Exact velocity gradient by the problem's hand-written derivatives."""
    _, grad, _, _ = prob._parts(x)
    return np.sin(t) * grad
