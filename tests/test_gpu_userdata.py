"""Problem data from the caller (stmg_set_data, stmg_initial_condition with a callback): the body
force f, the Dirichlet data g and the initial velocity v0 given as host functions (Sec. 2, Problem
2.1), evaluated by the library at the Gauss points of the finest mesh.

* a callback holding the Taylor-Green data reproduces the built-in TG2D residual, initial field and
  slab solve (same kernels; the data differ only by the host's and the device's rounding of the
  same formula);
* polynomial flows with nonzero f and g (2D and 3D, mapped meshes) match the oracle's residual,
  computed from the same data functions, to 1e-12 relative.
"""
import numpy as np
import pytest

from oracle import forms, problems
from oracle.mesh import Mesh, Space
from oracle.reference import TimeData
from paper_2602_13841_gb300 import inputs
from tests.helpers import build_and_load, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


def _tg_velocity(x, t, nu):
    """Taylor-Green velocity, x of shape (2, npts)."""
    F = np.exp(-2.0 * np.pi ** 2 * nu * t)
    return F * np.stack([np.sin(np.pi * x[0]) * np.cos(np.pi * x[1]), -np.cos(np.pi * x[0]) * np.sin(np.pi * x[1])])


def _solver(d, n, r, k, amp, seed, problem, nu=0.01, tau=0.05, **kw):
    from paper_2602_13841_gb300 import stmg
    build_and_load()
    verts = inputs.vertices(d, n, amp, seed)
    p = stmg.default_params(dim=d, n_cells_1d=n, r=r, k=k, nu=nu, tau=tau, problem=problem, **kw)
    return stmg.Solver(p, verts), verts


def _t(a):
    import torch
    return torch.tensor(a, dtype=torch.float64, device="cuda")


def test_taylor_green_callbacks_reproduce_the_builtin_problem():
    import torch
    d, n, r, k, nu = 2, 6, 2, 2, 0.01
    ref, _ = _solver(d, n, r, k, 0.1, 5, "TG2D", nu=nu)
    usr, _ = _solver(d, n, r, k, 0.1, 5, "TG2D", nu=nu)
    usr.set_data(f=None, g=lambda x, t: _tg_velocity(x, t, nu))
    L = ref.levels[0]
    # initial field
    V_ref = torch.empty(L["Nv"], dtype=torch.float64, device="cuda")
    V_usr = torch.empty_like(V_ref)
    ref.initial_condition(V_ref)
    usr.initial_condition(V_usr, v0=lambda x, t: _tg_velocity(x, 0.0, nu))
    torch.cuda.synchronize()
    assert float((V_ref - V_usr).abs().max()) <= 1e-14
    # residual at a random state, two slab start times (the tables follow t_start)
    U = _t(inputs.uniform(L["Nst"], 3))
    Vp = _t(inputs.uniform(L["Nv"], 4))
    for t0 in (0.0, 0.35):
        Ra = torch.empty(L["Nst"], dtype=torch.float64, device="cuda")
        Rb = torch.empty_like(Ra)
        ref.residual(t0, U, Vp, Ra)
        usr.residual(t0, U, Vp, Rb)
        torch.cuda.synchronize()
        err = float((Ra - Rb).abs().max() / Ra.abs().max())
        assert err < 1e-13, (t0, err)
    # slab solve from the initial field
    Ua = torch.empty(L["Nst"], dtype=torch.float64, device="cuda")
    Ub = torch.empty_like(Ua)
    ref.initial_guess(V_ref, Ua)
    usr.initial_guess(V_usr, Ub)
    _, sa = ref.slab_solve(0.0, V_ref, Ua)
    _, sb = usr.slab_solve(0.0, V_usr, Ub)
    torch.cuda.synchronize()
    assert sa["res_final"] <= 1e-8 * sa["res0"] or sa["res_final"] <= 1e-12
    assert sb["res_final"] <= 1e-8 * sb["res0"] or sb["res_final"] <= 1e-12
    assert float((Ua - Ub).abs().max() / Ua.abs().max()) < 1e-9


class _Poly2D(problems.Problem):
    """v = (1 + t)(y^2 + 0.3 x, x^2 - 0.3 y) (div-free), g = v, f = an arbitrary smooth field."""

    def v(self, x, t):
        X, Y = x[..., 0], x[..., 1]
        return (1.0 + t) * np.stack([Y * Y + 0.3 * X, X * X - 0.3 * Y], -1)

    def g(self, x, t):
        return self.v(x, t)

    def f(self, x, t):
        X, Y = x[..., 0], x[..., 1]
        return np.stack([np.cos(2 * X + t) * Y, np.sin(X * Y) + t * X], -1)


class _Poly3D(problems.Problem):
    """g = (1 + t)(y z, x z^2, 0.5 x y), f = an arbitrary smooth field."""

    def g(self, x, t):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return (1.0 + t) * np.stack([Y * Z, X * Z * Z, 0.5 * X * Y], -1)

    def f(self, x, t):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return np.stack([np.cos(X + t) * Z, Y * Y - t, np.sin(X * Z) + Y], -1)


def _as_callback(fun):
    """(d, npts) coordinates -> (d, npts) values from a function of (npts, d) points."""
    return lambda x, t: np.ascontiguousarray(fun(np.ascontiguousarray(x.T), t).T)


@pytest.mark.parametrize("d,n,r,k,amp", [(2, 5, 2, 1, 0.15), (2, 4, 1, 2, 0.1), (3, 3, 1, 1, 0.15),
                                         (3, 2, 2, 2, 0.1)])
def test_user_data_residual_matches_oracle(d, n, r, k, amp):
    import torch
    nu = 0.02
    S, verts = _solver(d, n, r, k, amp, 8, "TG2D" if d == 2 else "TG3D", nu=nu)
    prob = (_Poly2D if d == 2 else _Poly3D)(nu)
    S.set_data(f=_as_callback(prob.f), g=_as_callback(prob.g))
    sp = Space(Mesh(d, n, verts), r)
    td = TimeData(k, S.params.tau)
    lay = forms.SlabLayout(sp, k)
    U = inputs.uniform(lay.Nst, 6)
    Vp = inputs.uniform(lay.Nv, 7)
    for t0 in (0.2, 0.45):
        R_or = forms.residual(sp, td, U, Vp, prob, t0)
        R = torch.empty(lay.Nst, dtype=torch.float64, device="cuda")
        S.residual(t0, _t(U), _t(Vp), R)
        torch.cuda.synchronize()
        err = np.abs(R.cpu().numpy() - R_or).max() / np.abs(R_or).max()
        assert err < 1e-12, (t0, err)


def test_user_initial_condition_is_the_nodal_interpolant_3d():
    import torch
    d, n, r = 3, 3, 2
    S, verts = _solver(d, n, r, 1, 0.1, 9, "TG3D")
    prob = _Poly3D(0.01)
    V0 = torch.empty(S.levels[0]["Nv"], dtype=torch.float64, device="cuda")
    S.initial_condition(V0, v0=_as_callback(prob.g))
    sp = Space(Mesh(d, n, verts), r)
    want = forms.interpolate_velocity(sp, lambda x: prob.g(x, 0.0))
    torch.cuda.synchronize()
    assert np.abs(V0.cpu().numpy() - want).max() < 1e-14 * np.abs(want).max()
