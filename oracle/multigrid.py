"""hp space-time multigrid preconditioner (oracle; test infrastructure).

Sec. 4.2 (hierarchy, grid transfers, cycle and coarsening order) and Sec. 4.3 (inexact
space-time Vanka smoother), restated as plain assembled linear algebra:

* hierarchy: p-coarsening first -- the taller of the r / k hierarchies alone until the heights
  match, then both, degree halving -- then h-coarsening of the space mesh (every second
  vertex); the time mesh is never coarsened;
* prolongation P = E_time (x) P_space, the canonical embedding: a coarse function is evaluated
  at the fine nodes (velocity: fine Gauss-Lobatto nodes, reference-cell embedding for the
  children of a coarse cell; pressure: exact L2 re-expansion of the coarse polynomial in the
  fine Legendre modes; time: coarse Lagrange polynomial at the fine Radau points);
* restriction R = P^T;
* level state: the fine velocity evaluated at the coarse nodes and Radau points;
* level operator: the Jacobian rediscretised at the level state, with the finest level's
  Nitsche penalty length on every level (h_{Gamma_D} scaled by n_level / n_finest and the
  finest degree factor), which makes the penalty term of the level operator equal to its
  Galerkin product P^T A P on nested meshes; with the level's own h and degree the coarse
  penalty is too weak and the V-cycle diverges;
* Vanka (Eq. LVS, vanka0): additive over cells, damping omega = 1.2 / 2^d unless given, patch = all velocity and pressure DoFs of the
  cell at all time nodes, patch matrix = the global submatrix R_K J~ R_K^T of the midpoint
  surrogate J~ (Eq. DefTildeHn, DefVnAst), inverted by dense LU with partial pivoting;
* V-cycle with nu1 / nu2 sweeps; coarsest level: dense LU of the assembled Jacobian bordered by
  one mean-zero pressure row per time node (pure Dirichlet, L^2_0).
"""
import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import forms
from .mesh import Mesh, Space
from .reference import TimeData, gauss_lobatto_01, lagrange_eval, legendre01
from numpy.polynomial import legendre as npleg


def height(x):
    h = 0
    while x > 1:
        x //= 2
        h += 1
    return h


def hierarchy(d, n, r, k, vertices, max_h=-1, keep_k=False):
    """List of (n, r, k, vertices) from fine to coarse.  keep_k: p-coarsen in space only and keep
    DG(k) on every level (a variant of the paper's order, which halves k as well)."""
    levels = [(n, r, k, np.asarray(vertices, float))]
    while height(r) > 0 or (height(k) > 0 and not keep_k):
        if keep_k or height(r) > height(k):
            r //= 2
        elif height(k) > height(r):
            k //= 2
        else:
            r //= 2
            k //= 2
        levels.append((n, r, k, levels[-1][3]))
    hl = 0
    V = levels[-1][3]
    while n % 2 == 0 and n // 2 >= 2 and (max_h < 0 or hl < max_h):
        V = V.reshape(*([n + 1] * d), d)[tuple([slice(None, None, 2)] * d)].reshape(-1, d)
        n //= 2
        hl += 1
        levels.append((n, r, k, V))
    return levels


# ----------------------------------------------------------------------------- 1D operators
def _node_positions_1d(n, r):
    """Reference positions of the global 1D velocity nodes of an n-cell line (cell units)."""
    g = gauss_lobatto_01(r + 2)
    return np.array([c + g[i] for c in range(n) for i in range(r + 1)] + [float(n)])


def eval_1d(n, r, x):
    """E[p, j] = value at x_p (cell units) of the global 1D basis function j of the n-cell line."""
    x = np.asarray(x, float)
    N1 = (r + 1) * n + 1
    E = np.zeros((len(x), N1))
    g = gauss_lobatto_01(r + 2)
    for p, xp in enumerate(x):
        c = min(int(np.floor(xp)), n - 1)
        L = lagrange_eval(g, [xp - c])[0]
        E[p, c * (r + 1):c * (r + 1) + r + 2] = L
    return E


def velocity_prolongation(d, nf, rf, nc, rc):
    """P_space for one velocity component: coarse function at the fine nodes (tensor product)."""
    xf = _node_positions_1d(nf, rf) * (nc / nf)
    P1 = sp.csr_matrix(eval_1d(nc, rc, xf))
    P = P1
    for _ in range(d - 1):
        P = sp.kron(P1, P, format="csr")       # x fastest: last factor is the x direction
    return P


def velocity_interpolation(d, nf, rf, nc, rc):
    """Fine velocity evaluated at the coarse nodes (the level-state transfer)."""
    xc = _node_positions_1d(nc, rc) * (nf / nc)
    I1 = sp.csr_matrix(eval_1d(nf, rf, xc))
    I = I1
    for _ in range(d - 1):
        I = sp.kron(I1, I, format="csr")
    return I


def _legendre_child_1d(r, b):
    """T[i, j]: P_i(2 X - 1) with X = (b + x)/2 expanded in P_j(2x - 1) on [0,1] (exact)."""
    xg, wg = npleg.leggauss(r + 2)
    x = 0.5 * (xg + 1.0)
    w = 0.5 * wg
    Lc = legendre01(r, 0.5 * (b + x))             # coarse modes at child points
    Lf = legendre01(r, x)
    norms = 1.0 / (2 * np.arange(r + 1) + 1)
    return np.einsum("q,qi,qj->ij", w, Lc, Lf) / norms[None, :]


def pressure_prolongation(d, nf, rf, nc, rc, modes_f, modes_c):
    """Coarse P_rc^disc function re-expanded exactly in the fine P_rf modes of each fine cell."""
    npf, npc = len(modes_f), len(modes_c)
    rows, cols, vals = [], [], []
    cells_f = np.array(list(itertools.product(*([range(nf)] * d))))[:, ::-1]
    ratio = nf // nc
    Tch = {b: _legendre_child_1d(max(rf, rc), b) for b in (0, 1)}
    for cf, cm in enumerate(cells_f):
        cc = cm // ratio
        bits = cm % ratio
        ccidx = int(np.dot(cc, nc ** np.arange(d)))
        for i, mc in enumerate(modes_c):
            for j, mf in enumerate(modes_f):
                if ratio == 1:
                    v = 1.0 if tuple(mc) == tuple(mf) else 0.0
                else:
                    v = np.prod([Tch[bits[l]][mc[l], mf[l]] for l in range(d)])
                if v != 0.0:
                    rows.append(cf * npf + j)
                    cols.append(ccidx * npc + i)
                    vals.append(v)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf ** d * npf, nc ** d * npc))


def time_prolongation(kf, kc):
    """E[i, j] = phi^c_j(t_i^f): coarse DG(kc) polynomial at the fine Radau points."""
    tf = TimeData(kf, 1.0)
    tc = TimeData(kc, 1.0)
    return tc.eval_basis(tf.that)


class Level:
    def __init__(self, d, n, r, k, vertices, tau, nu, gamma=(10.0, 10.0), bconv=True, hscale=None):
        self.d, self.n, self.r, self.k = d, n, r, k
        self.hscale = hscale
        self.space = Space(Mesh(d, n, vertices), r)
        self.td = TimeData(k, tau)
        self.lay = forms.SlabLayout(self.space, k)
        self.nu, self.gamma, self.bconv = nu, gamma, bconv
        self.Nst = self.lay.Nst


def transfer(fine, coarse):
    """Slab prolongation P (coarse -> fine) and velocity state interpolation I (fine -> coarse)."""
    d = fine.d
    E = time_prolongation(fine.k, coarse.k)                    # [kf+1, kc+1]
    Pv1 = velocity_prolongation(d, fine.n, fine.r, coarse.n, coarse.r)
    Pv = sp.block_diag([Pv1] * d, format="csr")
    Pp = pressure_prolongation(d, fine.n, fine.r, coarse.n, coarse.r,
                               fine.space.ref.modes, coarse.space.ref.modes)
    P = sp.bmat([[sp.kron(E, Pv), None], [None, sp.kron(E, Pp)]], format="csr")
    Iv1 = velocity_interpolation(d, fine.n, fine.r, coarse.n, coarse.r)
    Iv = sp.block_diag([Iv1] * d, format="csr")
    Et = TimeData(fine.k, 1.0).eval_basis(TimeData(coarse.k, 1.0).that)   # [kc+1, kf+1]
    Ivel = sp.kron(Et, Iv, format="csr")
    return P, Ivel


def midpoint_velocity(level, U):
    """v* = sum_a phi_a(t*) V^a at the slab midpoint t* (Eq. DefVnAst)."""
    phi = level.td.eval_basis([0.0])[0]
    return sum(phi[a] * level.lay.v(U, a) for a in range(level.k + 1))


def patch_dofs(level, cell):
    lay, s = level.lay, level.space
    idx = [lay.voff(a) + s.cell_vdofs[cell] for a in range(level.k + 1)]
    idx += [lay.poff(a) + s.cell_pdofs[cell] for a in range(level.k + 1)]
    return np.concatenate(idx)


class Vanka:
    """Cell-wise space-time Vanka with midpoint-surrogate patch matrices (Sec. 4.3)."""

    surrogate = True          # patches of J~ (convection at v*); ExactVanka: patches of J itself

    def __init__(self, level, U, omega, omega_p=None):
        self.level, self.omega = level, omega
        self.omega_p = omega if omega_p is None else omega_p
        nv = (level.k + 1) * level.lay.Nv
        # relaxation per DoF: omega on the (overlapping) velocity DoFs, omega_p on the pressure
        # DoFs, each of which belongs to exactly one patch
        self.weights = np.where(np.arange(level.Nst) < nv, omega, self.omega_p)
        vstar = midpoint_velocity(level, U) if self.surrogate else None
        Jt = forms.jacobian(level.space, level.td, U, level.nu, *level.gamma, level.bconv, vstar=vstar,
                            hscale=level.hscale)
        Jt = Jt.tocsr()
        self.patches = []
        for c in range(level.space.mesh.ncells):
            idx = patch_dofs(level, c)
            S = self.patch_matrix(Jt[idx][:, idx].toarray())
            self.patches.append((idx, sla.lu_factor(S)))

    def patch_matrix(self, S):
        """The local matrix whose inverse the sweep applies: the surrogate patch itself."""
        return S

    def sweep(self, J, rhs, d):
        """d <- d + W sum_K R_K^T S~_K^{-1} R_K (rhs - J d) (Eq. vanka0); W = omega on velocity
        DoFs, omega_p on pressure DoFs (W = omega I when omega_p = omega)."""
        res = rhs - J @ d
        upd = np.zeros_like(d)
        for idx, lu in self.patches:
            upd[idx] += sla.lu_solve(lu, res[idx])
        return d + self.weights * upd


class ExactVanka(Vanka):
    """Space-time Vanka with the exact patch matrices R_K J R_K^T: the convection Jacobian of every
    time node at that node's own velocity V^a (Eq. JacobianLocal2), the matrix the midpoint
    surrogate of Sec. 4.3 approximates (the comparison of its Lemma)."""

    surrogate = False


class DiagonalVanka(Vanka):
    """Diagonal space-time Vanka, the cheaper smoother of the paper's closing section (diagonal
    Vanka of John 2000, carried to the space-time patch): the velocity block of the surrogate
    patch matrix keeps only the entries that couple a spatial velocity DoF with itself -- one
    (k+1) x (k+1) temporal block K^tau M_ii + W A_ii per spatial DoF -- while the pressure
    coupling W (x) B_K stays whole.  The modified patch is solved exactly (dense LU here; the
    device solves it through its pressure Schur complement).

    The patch ordering is that of patch_dofs: velocity [time node][component][node], then
    pressure; spatial velocity DoF of a patch row = its position modulo d * nloc."""

    def patch_matrix(self, S):
        ms_v = self.level.d * self.level.space.nloc
        nvp = (self.level.k + 1) * ms_v
        sid = np.arange(nvp) % ms_v
        S = S.copy()
        S[:nvp, :nvp] *= sid[:, None] == sid[None, :]
        return S


class CoarseSolver:
    """Dense LU of the Jacobian bordered by the mean-zero pressure rows of every time node."""

    def __init__(self, level, J):
        s, lay, k = level.space, level.lay, level.k
        w = np.einsum("kq,qm->km", s.JxW, s.ref.psi).ravel()
        C = np.zeros((k + 1, lay.Nst))
        for a in range(k + 1):
            C[a, lay.poff(a):lay.poff(a) + lay.Np] = w
        A = np.zeros((lay.Nst + k + 1, lay.Nst + k + 1))
        A[:lay.Nst, :lay.Nst] = J.toarray()
        A[:lay.Nst, lay.Nst:] = C.T
        A[lay.Nst:, :lay.Nst] = C
        self.n = lay.Nst
        self.lu = sla.lu_factor(A)

    def solve(self, r):
        rhs = np.concatenate([r, np.zeros(self.lu[0].shape[0] - self.n)])
        return sla.lu_solve(self.lu, rhs)[:self.n]


class Multigrid:
    """hp-STMG V-cycle: z = B^{-1} r on the finest level (Sec. 4.2)."""

    def __init__(self, d, n, r, k, vertices, tau, nu, omega=None, nu1=1, nu2=1, omega_p=1.0,
                 gamma=(10.0, 10.0), bconv=True, max_h=-1, keep_k=False, smoother="vanka", nu_tc=0):
        # Eq. vanka0 leaves omega open; the additive sum puts each velocity vertex in up to 2^d
        # patches, so the default damping is 1.2 / 2^d (0.3 in 2D, 0.15 in 3D)
        if omega is None:
            omega = 1.2 / 2 ** d
        p0 = r + 1
        self.levels = [Level(d, ln, lr, lk, lv, tau, nu, gamma, bconv, hscale=(ln / n) / (p0 * (p0 + 1)))
                       for ln, lr, lk, lv in hierarchy(d, n, r, k, vertices, max_h, keep_k)]
        self.P, self.I = [], []
        for f, c in zip(self.levels[:-1], self.levels[1:]):
            P, I = transfer(f, c)
            self.P.append(P)
            self.I.append(I)
        self.omega, self.omega_p, self.nu1, self.nu2 = omega, omega_p, nu1, nu2
        # nu_tc > 0: pre- and post-sweeps on the levels whose next level has a lower time degree
        self.nu_tc = nu_tc
        # "vanka": the midpoint-surrogate patches of Sec. 4.3; "diagonal": DiagonalVanka
        self.smoother_cls = {"vanka": Vanka, "diagonal": DiagonalVanka, "exact": ExactVanka}[smoother]

    def level_states(self, U):
        """Velocity state of every level (pressure entries zero) from the fine slab vector."""
        states = [U]
        for l, (f, c) in enumerate(zip(self.levels[:-1], self.levels[1:])):
            Vf = states[-1][:(f.k + 1) * f.lay.Nv]
            Uc = np.zeros(c.Nst)
            Uc[:(c.k + 1) * c.lay.Nv] = self.I[l] @ Vf
            states.append(Uc)
        return states

    def setup(self, U):
        """Level Jacobians, Vanka patches (smoother build) and the coarse factorisation at U."""
        self.states = self.level_states(U)
        self.J = [forms.jacobian(L.space, L.td, S, L.nu, *L.gamma, L.bconv, hscale=L.hscale)
                  for L, S in zip(self.levels, self.states)]
        self.smoothers = [self.smoother_cls(L, S, self.omega, self.omega_p)
                          for L, S in zip(self.levels[:-1], self.states[:-1])]
        self.coarse = CoarseSolver(self.levels[-1], self.J[-1])

    def vcycle(self, r, l=0):
        if l == len(self.levels) - 1:
            return self.coarse.solve(r)
        J, sm = self.J[l], self.smoothers[l]
        nu1, nu2 = self.nu1, self.nu2
        if self.nu_tc > 0 and self.levels[l + 1].k < self.levels[l].k:
            nu1 = nu2 = self.nu_tc
        d = np.zeros_like(r)
        for _ in range(nu1):
            d = sm.sweep(J, r, d)
        rc = self.P[l].T @ (r - J @ d)
        d = d + self.P[l] @ self.vcycle(rc, l + 1)
        for _ in range(nu2):
            d = sm.sweep(J, r, d)
        return d
