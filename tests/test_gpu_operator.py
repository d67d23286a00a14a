"""GPU parity of the matrix-free operator kernels against the FP64 oracle (through the C ABI).

* y = J_n(U) x: FP64 to 1e-12 relative (max-norm, relative to max|y|), FP32 to 2e-5;
* R_n(U; V_prev): FP64 to 1e-12 relative;
* every level of the hp hierarchy (p-coarsened tables, h-coarsened meshes);
* ragged colour classes (odd n), Cartesian and perturbed meshes, d = 2, 3, r = 1..3, k = 0..2;
* the full-size configuration of the benchmark (2D 256^2, r = 2, k = 2, perturbed) checked
  cell by cell on sampled cells against the oracle on the 5^d block around each cell.
"""
import numpy as np
import pytest

from oracle import forms, problems
from oracle.mesh import Mesh, Space
from oracle.reference import TimeData
from paper_2602_13841_gb300 import inputs
from tests.helpers import Block, build_and_load, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]

PROB = {2: "TG2D", 3: "MMS3D"}


def _solver(d, n, r, k, amp, seed, nu=0.01, tau=0.05, problem=None, **kw):
    import torch
    from paper_2602_13841_gb300 import stmg
    build_and_load()
    verts = inputs.vertices(d, n, amp, seed)
    p = stmg.default_params(dim=d, n_cells_1d=n, r=r, k=k, nu=nu, tau=tau,
                            problem=problem or PROB[d], **kw)
    return stmg.Solver(p, verts), verts


def _t(a, dtype=None):
    import torch
    return torch.tensor(a, dtype=dtype or torch.float64, device="cuda")


CASES = [
    (2, 5, 1, 1, 0.0), (2, 6, 2, 2, 0.15), (2, 3, 3, 0, 0.2), (2, 7, 2, 1, 0.1),
    (3, 3, 1, 2, 0.15), (3, 2, 2, 1, 0.0), (3, 3, 2, 0, 0.2), (3, 2, 3, 1, 0.1),
]


@pytest.mark.parametrize("d,n,r,k,amp", CASES)
def test_apply_fp64_and_fp32_match_oracle(d, n, r, k, amp):
    import torch
    from paper_2602_13841_gb300 import stmg
    S, verts = _solver(d, n, r, k, amp, seed=7)
    sp = Space(Mesh(d, n, verts), r)
    td = TimeData(k, S.params.tau)
    lay = forms.SlabLayout(sp, k)
    assert S.levels[0]["Nst"] == lay.Nst
    U = inputs.uniform(lay.Nst, 1)
    x = inputs.uniform(lay.Nst, 2)
    y_or = forms.jacobian(sp, td, U, S.params.nu) @ x
    y = torch.empty(lay.Nst, dtype=torch.float64, device="cuda")
    S.apply(_t(U), _t(x), y, 0, stmg.STMG_FP64)
    torch.cuda.synchronize()
    err = np.abs(y.cpu().numpy() - y_or).max() / np.abs(y_or).max()
    assert err < 1e-12, err
    y32 = torch.empty(lay.Nst, dtype=torch.float32, device="cuda")
    S.apply(_t(U, torch.float32), _t(x, torch.float32), y32, 0, stmg.STMG_FP32)
    torch.cuda.synchronize()
    err32 = np.abs(y32.double().cpu().numpy() - y_or).max() / np.abs(y_or).max()
    assert err32 < 2e-5, err32


@pytest.mark.parametrize("d,n,r,k,amp,pname", [(2, 5, 1, 1, 0.0, "TG2D"), (2, 6, 2, 2, 0.15, "MMS2D"),
                                               (3, 3, 1, 2, 0.15, "MMS3D"), (3, 3, 2, 1, 0.1, "TG3D"),
                                               (3, 3, 2, 2, 0.1, "CAV3D")])
def test_residual_matches_oracle(d, n, r, k, amp, pname):
    import torch
    S, verts = _solver(d, n, r, k, amp, seed=3, problem=pname)
    sp = Space(Mesh(d, n, verts), r)
    td = TimeData(k, S.params.tau)
    lay = forms.SlabLayout(sp, k)
    prob = problems.make(pname, S.params.nu)
    U = inputs.uniform(lay.Nst, 4)
    Vp = inputs.uniform(lay.Nv, 5)
    t0 = 0.3
    R_or = forms.residual(sp, td, U, Vp, prob, t0)
    R = torch.empty(lay.Nst, dtype=torch.float64, device="cuda")
    S.residual(t0, _t(U), _t(Vp), R)
    torch.cuda.synchronize()
    err = np.abs(R.cpu().numpy() - R_or).max() / np.abs(R_or).max()
    assert err < 1e-12, err


@pytest.mark.parametrize("d,pname", [(2, "TG2D"), (3, "TG3D"), (3, "CAV3D")])
def test_initial_condition_is_nodal_interpolant(d, pname):
    import torch
    n, r = 4, 2
    S, verts = _solver(d, n, r, 1, 0.1, seed=9, problem=pname)
    sp = Space(Mesh(d, n, verts), r)
    V0_or = forms.interpolate_velocity(sp, problems.make(pname, S.params.nu).v0)
    V0 = torch.empty(sp.Nv, dtype=torch.float64, device="cuda")
    S.initial_condition(V0)
    torch.cuda.synchronize()
    assert np.abs(V0.cpu().numpy() - V0_or).max() < 1e-14


def test_every_level_of_the_hierarchy_matches_oracle():
    import torch
    from paper_2602_13841_gb300 import stmg
    d, n, r, k = 2, 8, 2, 2
    S, verts = _solver(d, n, r, k, 0.15, seed=11)
    assert [(L["n"], L["r"], L["k"]) for L in S.levels] == [(8, 2, 2), (8, 1, 1), (4, 1, 1), (2, 1, 1)]
    V = verts
    nprev = n
    for lvl, L in enumerate(S.levels):
        while nprev > L["n"]:                       # coarse meshes: every second vertex
            V = V.reshape(nprev + 1, nprev + 1, d)[::2, ::2].reshape(-1, d)
            nprev //= 2
        sp = Space(Mesh(d, L["n"], V), L["r"])
        td = TimeData(L["k"], S.params.tau)
        U = inputs.uniform(L["Nst"], 20 + lvl)
        x = inputs.uniform(L["Nst"], 40 + lvl)
        hscale = (L["n"] / n) / ((r + 1) * (r + 2))        # every level keeps the finest penalty
        y_or = forms.jacobian(sp, td, U, S.params.nu, hscale=hscale) @ x
        y = torch.empty(L["Nst"], dtype=torch.float64, device="cuda")
        S.apply(_t(U), _t(x), y, lvl, stmg.STMG_FP64)
        torch.cuda.synchronize()
        assert np.abs(y.cpu().numpy() - y_or).max() < 1e-12 * np.abs(y_or).max()


def test_full_size_apply_and_residual_sampled_cells():
    """2D 256^2 perturbed (amp 0.1 h, seed 1234), Q3/P2/DG(2): the benchmark's configuration."""
    import torch
    from paper_2602_13841_gb300 import stmg
    d, n, r, k = 2, 256, 2, 2
    S, verts = _solver(d, n, r, k, 0.1, seed=1234, nu=1e-3, tau=0.05, problem="TG2D")
    L = S.levels[0]
    U = inputs.uniform(L["Nst"], 42)
    x = inputs.uniform(L["Nst"], 43)
    Vp = inputs.uniform(L["Nv"], 44)
    y = torch.empty(L["Nst"], dtype=torch.float64, device="cuda")
    S.apply(_t(U), _t(x), y, 0, stmg.STMG_FP64)
    R = torch.empty(L["Nst"], dtype=torch.float64, device="cuda")
    S.residual(0.1, _t(U), _t(Vp), R)
    torch.cuda.synchronize()
    y, R = y.cpu().numpy(), R.cpu().numpy()
    rng = np.random.default_rng(0)
    cells = [(0, 0), (n - 1, n - 1), (0, n - 1), (n // 2, 0)] + [tuple(rng.integers(0, n, 2)) for _ in range(8)]
    prob = problems.make("TG2D", 1e-3)
    for cell in cells:
        B = Block(d, n, r, k, verts, list(cell))
        td = TimeData(k, 0.05)
        Ub, xb = U[B.slab_map], x[B.slab_map]
        yb = forms.jacobian(B.space, td, Ub, 1e-3) @ xb
        got = y[B.slab_map[B.rows]]
        want = yb[B.rows]
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), cell
        Rb = forms.residual(B.space, td, Ub, Vp[B.vel_map], prob, 0.1)
        got = R[B.slab_map[B.rows]]
        want = Rb[B.rows]
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), cell


@pytest.mark.parametrize("d,n,r,k,amp,nu,tau,pname", [
    (3, 64, 2, 1, 0.0, 1.0 / 1600, 0.02, "TG3D"),    # 3D 64^3 Cartesian, Q3/P2, DG(1), Re 1600
    (3, 128, 1, 2, 0.1, 1.0 / 400, 0.01, "MMS3D"),   # 3D 128^3 mapped, Q2/P1, DG(2), Re 400
])
def test_full_size_3d_apply_and_residual_sampled_cells(d, n, r, k, amp, nu, tau, pname):
    """The 3D workloads at full size: Jacobian apply and residual on the whole mesh, checked on
    sampled cells (a corner, a boundary-face cell, an interior cell) against the oracle on the
    5^3 block around each."""
    import torch
    from paper_2602_13841_gb300 import stmg
    S, verts = _solver(d, n, r, k, amp, seed=1234, nu=nu, tau=tau, problem=pname)
    L = S.levels[0]
    U = inputs.uniform(L["Nst"], 52)
    x = inputs.uniform(L["Nst"], 53)
    Vp = inputs.uniform(L["Nv"], 54)
    y = torch.empty(L["Nst"], dtype=torch.float64, device="cuda")
    S.apply(_t(U), _t(x), y, 0, stmg.STMG_FP64)
    R = torch.empty(L["Nst"], dtype=torch.float64, device="cuda")
    S.residual(0.3, _t(U), _t(Vp), R)
    torch.cuda.synchronize()
    y, R = y.cpu().numpy(), R.cpu().numpy()
    rng = np.random.default_rng(1)
    cells = [(0, 0, 0), (n // 2, 0, n // 3), tuple(int(c) for c in rng.integers(1, n - 1, 3))]
    if r >= 2:                      # the oracle's Q3 block takes ~20 s per assembly: two cells
        cells = [cells[0], cells[2]]
    prob = problems.make(pname, nu)
    td = TimeData(k, tau)
    for cell in cells:
        B = Block(d, n, r, k, verts, list(cell))
        Ub, xb = U[B.slab_map], x[B.slab_map]
        yb = forms.jacobian(B.space, td, Ub, nu) @ xb
        got, want = y[B.slab_map[B.rows]], yb[B.rows]
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), cell
        Rb = forms.residual(B.space, td, Ub, Vp[B.vel_map], prob, 0.3)
        got, want = R[B.slab_map[B.rows]], Rb[B.rows]
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), cell
