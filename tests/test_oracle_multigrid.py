"""Pins of the oracle's hp-STMG pieces (Sec. 4.2-4.3) against facts that do not come from the
oracle itself:

* canonical-embedding prolongation: a polynomial that the coarse space holds is reproduced
  exactly at the fine nodes (velocity: tensor polynomials of degree r_c + 1 on GLL nodes placed
  from the closed-form Gauss-Lobatto points; pressure: coarse modal functions evaluated at random
  points of the fine cells; time: polynomials of degree k_c at the Radau points);
* state interpolation: a fine polynomial evaluated at the coarse nodes;
* Galerkin identity: on nested Cartesian meshes at zero state, the rediscretised level operator
  equals P^T J_fine P exactly (mass, viscous, pressure, Nitsche terms are all integrated exactly
  and the coarse levels carry the finest Nitsche length) -- a transposed, mis-scaled or
  mis-ordered transfer, or a wrong coarse penalty, breaks it;
* coarse solve: for r in the range of J it returns x with J x = r and zero pressure mean;
* the V-cycle as a stationary iteration contracts the residual (2D and 3D, default damping).
"""
import itertools

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import forms, multigrid
from oracle.reference import TimeData, gauss_lobatto_01, pressure_modes
from paper_2602_13841_gb300 import inputs


def _grid_positions(n, r):
    """Global 1D GLL node positions of an n-cell Q_{r+1} line in [0, 1] (closed-form nodes)."""
    g = gauss_lobatto_01(r + 2)
    return np.array([(c + g[i]) / n for c in range(n) for i in range(r + 1)] + [1.0])


def _tensor_values(d, x1, f):
    """f at the tensor grid x1^d, x fastest (lexicographic node order of the slab layout)."""
    pts = np.array(list(itertools.product(*([x1] * d))))[:, ::-1]
    return f(pts)


def _poly(d, deg, seed):
    rng = np.random.default_rng(seed)
    exps = [e for e in itertools.product(range(deg + 1), repeat=d)]
    coef = rng.standard_normal(len(exps))

    def f(p):
        return sum(c * np.prod([p[:, l] ** e[l] for l in range(d)], axis=0) for c, e in zip(coef, exps))
    return f


@pytest.mark.parametrize("d,nf,rf,nc,rc", [(2, 4, 2, 4, 1), (2, 4, 1, 2, 1), (2, 6, 3, 6, 1), (3, 2, 2, 2, 1),
                                           (3, 4, 1, 2, 1)])
def test_velocity_prolongation_reproduces_coarse_polynomials(d, nf, rf, nc, rc):
    f = _poly(d, rc + 1, 3)
    vc = _tensor_values(d, _grid_positions(nc, rc), f)
    vf = _tensor_values(d, _grid_positions(nf, rf), f)
    P = multigrid.velocity_prolongation(d, nf, rf, nc, rc)
    assert np.abs(P @ vc - vf).max() < 1e-12 * np.abs(vf).max()


@pytest.mark.parametrize("d,nf,rf,nc,rc", [(2, 4, 2, 4, 1), (2, 4, 1, 2, 1), (3, 2, 2, 2, 1), (3, 4, 1, 2, 1)])
def test_velocity_state_interpolation_evaluates_fine_polynomials(d, nf, rf, nc, rc):
    f = _poly(d, rf + 1, 4)
    vf = _tensor_values(d, _grid_positions(nf, rf), f)
    vc = _tensor_values(d, _grid_positions(nc, rc), f)
    I = multigrid.velocity_interpolation(d, nf, rf, nc, rc)
    assert np.abs(I @ vf - vc).max() < 1e-12 * np.abs(vc).max()


def _eval_pressure(d, n, r, coef, pts):
    """Modal P_r^disc function (cell-major, x-fastest cells) at global points of [0,1]^d."""
    modes = pressure_modes(r, d)
    out = np.zeros(len(pts))
    for q, x in enumerate(pts):
        cell = np.minimum((x * n).astype(int), n - 1)
        xi = x * n - cell
        c = int(np.dot(cell, n ** np.arange(d)))
        for m, deg in enumerate(modes):
            val = 1.0
            for l in range(d):
                e = np.zeros(deg[l] + 1)
                e[deg[l]] = 1.0
                val *= npleg.legval(2.0 * xi[l] - 1.0, e)
            out[q] += coef[c * len(modes) + m] * val
    return out


@pytest.mark.parametrize("d,nf,rf,nc,rc", [(2, 4, 2, 4, 1), (2, 4, 1, 2, 1), (2, 4, 3, 2, 1), (3, 2, 2, 2, 1),
                                           (3, 4, 1, 2, 1)])
def test_pressure_prolongation_is_exact_reexpansion(d, nf, rf, nc, rc):
    mf, mc = pressure_modes(rf, d), pressure_modes(rc, d)
    rng = np.random.default_rng(11)
    coef_c = rng.standard_normal(nc ** d * len(mc))
    P = multigrid.pressure_prolongation(d, nf, rf, nc, rc, mf, mc)
    coef_f = P @ coef_c
    pts = rng.uniform(0.0, 1.0, size=(60, d))
    want = _eval_pressure(d, nc, rc, coef_c, pts)
    got = _eval_pressure(d, nf, rf, coef_f, pts)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("kf,kc", [(2, 1), (1, 0), (2, 0), (1, 1)])
def test_time_prolongation_reproduces_coarse_polynomials(kf, kc):
    tf, tc = TimeData(kf, 1.0), TimeData(kc, 1.0)
    c = np.random.default_rng(kf * 10 + kc).standard_normal(kc + 1)
    g = lambda t: np.polyval(c, t)
    E = multigrid.time_prolongation(kf, kc)
    assert np.abs(E @ g(tc.that) - g(tf.that)).max() < 1e-13


@pytest.mark.parametrize("d,n,r,k", [(2, 4, 1, 1), (2, 4, 2, 2), (2, 4, 3, 1), (3, 2, 2, 0), (3, 4, 1, 1)])
def test_galerkin_identity_on_nested_cartesian_meshes(d, n, r, k):
    verts = inputs.vertices(d, n, 0.0, 1)
    mg = multigrid.Multigrid(d, n, r, k, verts, 0.05, 1e-2)
    mg.setup(np.zeros(mg.levels[0].Nst))
    assert len(mg.levels) >= 2
    for l in range(len(mg.levels) - 1):
        G = (mg.P[l].T @ mg.J[l] @ mg.P[l]).toarray()
        C = mg.J[l + 1].toarray()
        assert np.abs(G - C).max() < 1e-12 * np.abs(C).max(), l


@pytest.mark.parametrize("d,n,r,k,amp", [(2, 2, 1, 1, 0.1), (2, 4, 2, 0, 0.0), (3, 2, 1, 1, 0.1)])
def test_coarse_solve_inverts_on_the_range(d, n, r, k, amp):
    verts = inputs.vertices(d, n, amp, 2)
    mg = multigrid.Multigrid(d, n, r, k, verts, 0.05, 1e-2, max_h=0)
    L = mg.levels[-1]
    mg.setup(inputs.uniform(mg.levels[0].Nst, 3))
    J = mg.J[-1]
    y = inputs.uniform(L.Nst, 4)
    rhs = J @ y
    x = mg.coarse.solve(rhs)
    assert np.abs(J @ x - rhs).max() < 1e-10 * np.abs(rhs).max()
    w = np.einsum("kq,qm->km", L.space.JxW, L.space.ref.psi).ravel()
    for a in range(k + 1):
        P = x[L.lay.poff(a):L.lay.poff(a) + L.lay.Np]
        assert abs(np.dot(w, P)) < 1e-10 * np.abs(P).max()


@pytest.mark.parametrize("d,n,r,k,nu,rate", [(2, 8, 1, 1, 1e-2, 0.45), (2, 8, 2, 2, 1e-3, 0.6),
                                              (3, 4, 1, 1, 1e-2, 0.7)])
def test_vcycle_iteration_contracts(d, n, r, k, nu, rate):
    """x <- x + B^{-1}(b - J x) at a smooth state (the interpolated Taylor-Green field at every
    time node): the residual falls at least by `rate` per cycle on average over 6 cycles."""
    from oracle import problems
    verts = inputs.vertices(d, n, 0.1, 9)
    mg = multigrid.Multigrid(d, n, r, k, verts, 0.05, nu)
    L = mg.levels[0]
    prob = problems.make("TG2D" if d == 2 else "TG3D", nu)
    V = forms.interpolate_velocity(L.space, prob.v0)
    U = np.concatenate([np.tile(V, k + 1), np.zeros((k + 1) * L.lay.Np)])
    mg.setup(U)
    J = mg.J[0]
    b = J @ inputs.uniform(L.Nst, 6)
    x = np.zeros(L.Nst)
    r0 = np.linalg.norm(b)
    for _ in range(6):
        x = x + mg.vcycle(b - J @ x)
    red = (np.linalg.norm(b - J @ x) / r0) ** (1.0 / 6.0)
    assert red < rate, red


def test_hierarchy_follows_the_coarsening_order():
    """Sec. 4.2: p first, (k, r) -> (k/2, r/2) with the taller hierarchy alone until the heights
    match, then h down to two cells per direction; keep_k (a variant) halves r only."""
    V = inputs.vertices(2, 8, 0.0, 1)
    rk = lambda lv: [(n, r, k) for n, r, k, _ in lv]
    assert rk(multigrid.hierarchy(2, 8, 2, 2, V)) == [(8, 2, 2), (8, 1, 1), (4, 1, 1), (2, 1, 1)]
    assert rk(multigrid.hierarchy(2, 8, 3, 1, V)) == [(8, 3, 1), (8, 1, 1), (4, 1, 1), (2, 1, 1)]
    assert rk(multigrid.hierarchy(2, 8, 1, 2, V)) == [(8, 1, 2), (8, 1, 1), (4, 1, 1), (2, 1, 1)]
    assert rk(multigrid.hierarchy(2, 8, 2, 2, V, keep_k=True)) == [(8, 2, 2), (8, 1, 2), (4, 1, 2), (2, 1, 2)]
    assert rk(multigrid.hierarchy(2, 8, 1, 2, V, keep_k=True)) == [(8, 1, 2), (4, 1, 2), (2, 1, 2)]


def test_vcycle_with_space_only_p_coarsening_contracts():
    """The variant hierarchy (DG(2) on every level) as a stationary iteration: the Galerkin
    identity holds on it too, and it contracts at least as fast as the paper's order here."""
    from oracle import problems
    d, n, r, k, nu = 2, 8, 2, 2, 1e-3
    verts = inputs.vertices(d, n, 0.1, 9)
    prob = problems.make("TG2D", nu)
    red = {}
    for keep in (False, True):
        mg = multigrid.Multigrid(d, n, r, k, verts, 0.05, nu, keep_k=keep)
        L = mg.levels[0]
        V = forms.interpolate_velocity(L.space, prob.v0)
        mg.setup(np.concatenate([np.tile(V, k + 1), np.zeros((k + 1) * L.lay.Np)]))
        J = mg.J[0]
        b = J @ inputs.uniform(L.Nst, 6)
        x = np.zeros(L.Nst)
        for _ in range(6):
            x = x + mg.vcycle(b - J @ x)
        red[keep] = (np.linalg.norm(b - J @ x) / np.linalg.norm(b)) ** (1.0 / 6.0)
    assert red[True] < 0.6 and red[True] <= red[False] * 1.05, red


def test_midpoint_surrogate_error_is_first_order_in_tau():
    """Lemma (local Vanka surrogate, Sec. 4.3): with a state that varies smoothly in time,
    ||S~ - S|| <= C tau with C proportional to ||M^tau||, so ||S~ - S|| / ||M^tau|| halves with
    tau; and ||I - S^{-1} S~|| <= ||S^{-1}|| ||S~ - S|| (item (ii)).  S, S~: the space-time
    patch matrices of one interior cell built from the exact Jacobian (convection at every time
    node) and from the midpoint surrogate."""
    from oracle import problems
    from oracle.mesh import Mesh, Space
    d, n, r, k, t0 = 2, 4, 1, 2, 0.7
    verts = inputs.vertices(d, n, 0.1, 3)
    prob = problems.make("MMS2D", 1e-2)
    s = Space(Mesh(d, n, verts), r)
    cell = 5                                                   # interior cell (1, 1)
    ratios = []
    for tau in (0.2, 0.1, 0.05, 0.025):
        L = multigrid.Level(d, n, r, k, verts, tau, prob.nu, hscale=None)
        times = L.td.times(t0)
        U = np.concatenate([np.concatenate([forms.interpolate_velocity(s, lambda x, t=t: prob.v(x, t))
                                            for t in times]), np.zeros((k + 1) * L.lay.Np)])
        J = forms.jacobian(L.space, L.td, U, prob.nu)
        Jt = forms.jacobian(L.space, L.td, U, prob.nu, vstar=multigrid.midpoint_velocity(L, U))
        idx = multigrid.patch_dofs(L, cell)
        S = J[idx][:, idx].toarray()
        E = Jt[idx][:, idx].toarray() - S
        nE = np.linalg.norm(E, 2)
        ratios.append(nE / np.linalg.norm(L.td.M, 2))
        lhs = np.linalg.norm(np.eye(len(idx)) - np.linalg.solve(S, S + E), 2)
        assert lhs <= np.linalg.norm(np.linalg.inv(S), 2) * nE * (1 + 1e-12)
    rates = [ratios[i] / ratios[i + 1] for i in range(len(ratios) - 1)]
    assert all(1.8 < q < 2.2 for q in rates[1:]), (ratios, rates)


def test_two_grid_diverges_for_an_unresolved_convective_flow():
    """A limit of the method as read, recorded in the design notes: on 2D 32^2 Q2/P1 DG(0) at
    Re 1623 (dt = 0.05) the two-grid error propagation I - B^{-1} J (one h-level, one sweep) grows
    for the Taylor-Green state while it contracts for the manufactured solution at the same Re
    and mesh.  Power iteration from a seeded vector, mean-zero pressure kept."""
    from oracle import krylov, problems
    out = {}
    for pname in ("TG2D", "MMS2D"):
        prob = problems.make(pname, 1.0 / 1623.0)
        S = krylov.SlabSolver(2, 32, 1, 0, inputs.vertices(2, 32, 0.1, 1), 0.05, prob, max_h=1)
        L = S.L
        V = forms.interpolate_velocity(L.space, prob.v0)
        U = np.concatenate([V, np.zeros(L.lay.Np)])
        S.mg.setup(U)
        J = forms.jacobian(L.space, L.td, U, prob.nu)
        e = S.project(np.random.default_rng(0).standard_normal(L.Nst))
        e /= np.linalg.norm(e)
        growth = []
        for _ in range(12):
            e = S.project(e - S.mg.vcycle(J @ e))
            growth.append(np.linalg.norm(e))
            e /= growth[-1]
        out[pname] = float(np.exp(np.mean(np.log(growth[-5:]))))
    assert out["TG2D"] > 2.0, out
    assert out["MMS2D"] < 0.7, out


def test_time_p_coarsening_amplifies_smooth_errors_in_the_dropped_temporal_mode():
    """The mechanism behind the FGMRES counts of the paper's coarsening order (the design notes'
    reading on time p-coarsening): on 2D 8^2 Q3/P2 DG(2) (Taylor-Green state, Re 100, tau = h) an
    error that is smooth in space and lies in the temporal mode that DG(2) -> DG(1) drops (the
    Legendre polynomial of degree 2 at the Radau nodes) grows in the first V-cycle when the time
    degree is coarsened, and contracts when DG(2) is kept on every level; errors in the lowest
    temporal mode contract with both hierarchies."""
    from numpy.polynomial import legendre as npleg
    from oracle import problems
    from oracle.reference import radau_right
    d, n, r, k, nu = 2, 8, 2, 2, 1e-2
    first = {}
    for keep in (False, True):
        mg = multigrid.Multigrid(d, n, r, k, inputs.vertices(d, n, 0.0, 1), 1.0 / n, nu, keep_k=keep)
        L = mg.levels[0]
        prob = problems.make("TG2D", nu)
        V = forms.interpolate_velocity(L.space, prob.v0)
        U = np.concatenate([np.tile(V, k + 1), np.zeros((k + 1) * L.lay.Np)])
        mg.setup(U)
        J = mg.J[0]
        X = L.space.node_coords()
        smooth = np.sin(np.pi * X[:, 0]) * np.sin(np.pi * X[:, 1])
        that, _ = radau_right(k)
        for deg in (0, k):
            q = npleg.legval(that, [0] * deg + [1])
            e = np.zeros(L.Nst)
            for a in range(k + 1):
                e[a * L.lay.Nv:a * L.lay.Nv + d * len(smooth)] = q[a] * np.tile(smooth, d)
            first[(keep, deg)] = np.linalg.norm(e - mg.vcycle(J @ e)) / np.linalg.norm(e)
    assert first[(False, k)] > 1.5, first          # paper's order: amplified
    assert first[(True, k)] < 0.5, first           # DG(2) kept: contracted
    assert first[(False, 0)] < 0.5 and first[(True, 0)] < 0.5, first


def _slowest_mode(keep_k, nu_tc=0, d=2, n=8, r=1, k=2, nu=1e-2):
    """Power iteration on the V-cycle error propagation I - B^{-1} J with the constant pressure of
    every time node projected out: the geometric-mean growth of the last 20 of 60 steps, the
    pressure share of the limiting vector, and the shares of its pressure in the temporal Legendre
    modes of degree 0 .. k."""
    from numpy.polynomial import legendre as npleg
    from oracle import krylov, problems
    from oracle.reference import radau_right
    prob = problems.make("TG2D", nu)
    S = krylov.SlabSolver(d, n, r, k, inputs.vertices(d, n, 0.0, 1), 1.0 / n, prob, keep_k=keep_k, nu_tc=nu_tc)
    L, mg = S.L, S.mg
    V = forms.interpolate_velocity(L.space, prob.v0)
    U = np.concatenate([np.tile(V, k + 1), np.zeros((k + 1) * L.lay.Np)])
    mg.setup(U)
    J = mg.J[0]
    e = S.project(np.random.default_rng(0).standard_normal(L.Nst))
    e /= np.linalg.norm(e)
    growth = []
    for _ in range(60):
        e = S.project(e - mg.vcycle(J @ e))
        growth.append(np.linalg.norm(e))
        e /= growth[-1]
    nv, npr = L.lay.Nv, L.lay.Np
    that, _ = radau_right(k)
    Q = np.stack([npleg.legval(that, [0] * g + [1]) for g in range(k + 1)])
    pres = np.stack([e[(k + 1) * nv + a * npr:(k + 1) * nv + (a + 1) * npr] for a in range(k + 1)])
    modal = np.sum((np.linalg.inv(Q.T) @ pres) ** 2, axis=1)
    return (float(np.exp(np.mean(np.log(growth[-20:])))), float(np.linalg.norm(e[(k + 1) * nv:]) ** 2),
            modal / modal.sum())


def test_time_p_coarsening_leaves_smooth_pressure_errors_in_the_dropped_temporal_mode():
    """The cause of the FGMRES counts of the paper's coarsening order (the design notes' reading
    on time p-coarsening), on 2D 8^2 Q2/P1 DG(2) (Taylor-Green state, Re 100, tau = h): with
    DG(2) -> DG(1) the slowest error of the V-cycle is a pressure error, mostly in the temporal
    mode that DG(1) cannot represent, and it contracts by only about 0.96 per cycle; extra sweeps
    on the DG(2) level help a little; with DG(2) kept on every level the slowest error contracts
    by about 0.56."""
    rate, pshare, modal = _slowest_mode(False)
    assert rate > 0.93 and pshare > 0.95 and modal[2] > 0.5, (rate, pshare, modal)
    rate5 = _slowest_mode(False, nu_tc=5)[0]
    assert rate5 < rate - 0.03, (rate5, rate)
    rate_keep = _slowest_mode(True)[0]
    assert rate_keep < 0.65, rate_keep
