"""Pins of the oracle's lid-driven cavity data (Sec. 5.2) against facts that do not come from the
oracle:

* at zero state and zero previous-slab velocity the residual is minus the Nitsche data term of
  the lid.  The lid velocity is tangential (g.n = 0), so the pressure rows and the y- and
  z-velocity rows vanish and only nodes of the top cell layer are touched; the basis functions of
  a cell sum to one, so the consistency term (grad z . n) g drops out of the sum of the x-rows,
  which is then -w_a nu gamma_1 sin(pi t_a / 4) sum_F |F| / h_F with t_a, w_a the right Radau
  points and weights (closed forms) mapped to the slab and h_F = (|K| / |F|) / (p (p + 1)) the
  degree-scaled Nitsche length (p = r + 1).  A lid on the wrong face or component, a wrong time
  profile or a missing slab weight breaks it;
* the slab solution on a Cartesian mesh is mirror symmetric in y (the data are): v_x, v_z and p
  even, v_y odd, pressure modes of odd y-degree odd.
"""
import numpy as np
import pytest

from oracle import forms, krylov, problems
from oracle.mesh import Mesh, Space, uniform_vertices
from oracle.reference import TimeData, pressure_modes

# right Radau points and weights on [-1, 1] (the right end point included), k + 1 points
RADAU = {1: ([-1.0 / 3.0, 1.0], [1.5, 0.5]),
         2: ([(-1 - 6 ** 0.5) / 5, (-1 + 6 ** 0.5) / 5, 1.0], [(16 - 6 ** 0.5) / 18, (16 + 6 ** 0.5) / 18, 2.0 / 9.0])}


def test_lid_data_values():
    prob = problems.make("CAV3D", 4e-4)
    x = np.array([[0.3, 0.7, 1.0], [0.3, 0.7, 0.0], [1.0, 0.2, 0.9999], [0.5, 0.5, 0.5]])
    g = prob.g(x, 2.0)
    assert np.array_equal(g[0], [1.0, 0.0, 0.0])                 # sin(pi/2) on the lid
    assert np.abs(g[1:]).max() == 0.0
    assert np.abs(prob.v0(x)).max() == 0.0 and np.abs(prob.f(x, 1.0)).max() == 0.0


@pytest.mark.parametrize("n,r,k,t0,tau", [(2, 1, 1, 0.3, 0.25), (3, 2, 2, 1.1, 0.5)])
def test_zero_state_residual_is_the_lid_term(n, r, k, t0, tau):
    nu, gamma1 = 4e-4, 10.0
    s = Space(Mesh(3, n, uniform_vertices(3, n)), r)
    td = TimeData(k, tau)
    lay = forms.SlabLayout(s, k)
    prob = problems.make("CAV3D", nu)
    R = forms.residual(s, td, np.zeros(lay.Nst), np.zeros(lay.Nv), prob, t0)
    N1 = n * (r + 1) + 1
    z_index = np.arange(N1 ** 3) // (N1 * N1)                  # node (ix, iy, iz), x fastest
    top_layer = z_index >= N1 - 1 - (r + 1)
    p = r + 1
    h = (1.0 / n) / (p * (p + 1))                              # |K| / |F| = 1/n, scaled
    area = 1.0                                                 # sum of the lid faces' areas
    that, what = RADAU[k]
    for a in range(k + 1):
        V = lay.v(R, a)
        Rx, Ry, Rz = V[:N1 ** 3], V[N1 ** 3:2 * N1 ** 3], V[2 * N1 ** 3:]
        assert np.abs(lay.p(R, a)).max() == 0.0
        assert np.abs(Ry).max() == 0.0 and np.abs(Rz).max() == 0.0
        assert np.abs(Rx[~top_layer]).max() == 0.0
        ta = t0 + 0.5 * tau * (that[a] + 1.0)
        wa = 0.5 * tau * what[a]
        want = -wa * nu * gamma1 * np.sin(np.pi * ta / 4.0) * area / h
        assert abs(Rx.sum() - want) < 1e-12 * abs(want)


def _mirror_y(lay, s, n, r, k, U):
    """The slab vector of the solution mirrored at y = 1/2."""
    N1 = n * (r + 1) + 1
    ix, iy, iz = np.meshgrid(np.arange(N1), np.arange(N1), np.arange(N1), indexing="ij")
    node = (ix + N1 * (iy + N1 * iz)).ravel()
    image = (ix + N1 * ((N1 - 1 - iy) + N1 * iz)).ravel()
    modes = pressure_modes(r, 3)
    sign = np.array([(-1.0) ** m[1] for m in modes])
    cx, cy, cz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cell = (cx + n * (cy + n * cz)).ravel()
    cimage = (cx + n * ((n - 1 - cy) + n * cz)).ravel()
    W = np.zeros_like(U)
    for a in range(k + 1):
        V, Vw = lay.v(U, a), np.zeros(lay.Nv)
        for c, parity in enumerate((1.0, -1.0, 1.0)):
            Vw[c * N1 ** 3 + node] = parity * V[c * N1 ** 3 + image]
        P = lay.p(U, a).reshape(n ** 3, len(modes))
        Pw = np.zeros_like(P)
        Pw[cell] = P[cimage] * sign
        W[lay.voff(a):lay.voff(a) + lay.Nv] = Vw
        W[lay.poff(a):lay.poff(a) + lay.Np] = Pw.ravel()
    return W


def test_slab_solution_is_mirror_symmetric_in_y():
    n, r, k, tau, t0 = 2, 1, 1, 0.25, 1.0
    prob = problems.make("CAV3D", 1e-2)
    S = krylov.SlabSolver(3, n, r, k, uniform_vertices(3, n), tau, prob, rtol=1e-12, atol=0.0)
    L = S.L
    U0 = np.zeros(L.Nst)
    X, st = S.solve(U0, np.zeros(L.lay.Nv), t0)
    assert st.res <= 1e-12 * st.res0
    W = _mirror_y(L.lay, L.space, n, r, k, X)
    nv = (k + 1) * L.lay.Nv
    scale = np.abs(X[:nv]).max()
    assert scale > 0.05                                          # the lid drives a flow
    assert np.abs(W - X).max() < 1e-9 * max(scale, np.abs(X[nv:]).max())


def test_space_time_size_matches_the_papers_table():
    """Table st-sizes, c = 4, r = 2: 16^3 cells, 256 slabs of DG(2) on [0, 8], Q3/P2disc --
    302 520 576 space-time unknowns; the oracle's slab layout times the number of slabs."""
    s = Space(Mesh(3, 16, uniform_vertices(3, 16)), 2)
    lay = forms.SlabLayout(s, 2)
    assert 256 * lay.Nst == 302520576
