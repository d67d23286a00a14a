"""GPU parity of the hp-STMG preconditioner and the Newton-FGMRES slab solve (through the C ABI).

Against the oracle (same seeded inputs, FP64 preconditioner on the GPU unless stated):
* prolongation, restriction and state interpolation of every level pair: 1e-13 relative;
* the level states of a smoother build: 1e-13 relative;
* Vanka sweeps (from zero and from a nonzero iterate) on every smoothed level: 1e-9 relative
  (the patch inverses are Gauss-Jordan on the GPU, LU on the oracle; patches are ill-conditioned);
* one V-cycle: 1e-8 relative (coarse solve: FP32 inverse plus FP64 iterative refinement);
* slab solves reach the Newton tolerance, and the GPU solution (FP64 or FP32 preconditioner)
  equals the exact discrete solution (oracle Newton with sparse direct solves) to 1e-7 relative.
"""
import numpy as np
import pytest

from oracle import forms, marching, multigrid, problems
from oracle.reference import TimeData
from paper_2602_13841_gb300 import inputs
from tests.helpers import build_and_load, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


def _t(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), dtype=dtype or torch.float64, device="cuda")


def _np(t):
    return t.double().cpu().numpy()


def _setup(d, n, r, k, amp, precision="fp64", omega=None, nu=0.01, tau=0.05, problem="TG2D", seed=5, **kw):
    from paper_2602_13841_gb300 import stmg
    build_and_load()
    verts = inputs.vertices(d, n, amp, seed)
    prec = stmg.STMG_FP64 if precision == "fp64" else stmg.STMG_FP32
    p = stmg.default_params(dim=d, n_cells_1d=n, r=r, k=k, nu=nu, tau=tau, problem=problem,
                            omega=omega or 0.0, precond_precision=prec, **kw)
    S = stmg.Solver(p, verts)
    mg = multigrid.Multigrid(d, n, r, k, verts, tau, nu, omega=omega, keep_k=bool(kw.get("keep_time_degree", 0)))
    return S, mg, verts


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("d,n,r,k,amp,prec", [(2, 8, 2, 2, 0.15, "fp64"), (2, 6, 3, 1, 0.0, "fp64"),
                                              (3, 4, 1, 1, 0.1, "fp32"), (3, 4, 2, 1, 0.1, "fp32")])
def test_transfers_match_oracle(d, n, r, k, amp, prec):
    import torch
    S, mg, _ = _setup(d, n, r, k, amp, precision=prec)
    tol = 1e-13 if prec == "fp64" else 2e-6
    dt = S.pdtype
    assert [(L["n"], L["r"], L["k"]) for L in S.levels] == [(L.n, L.r, L.k) for L in mg.levels]
    for l in range(len(mg.levels) - 1):
        f, c = mg.levels[l], mg.levels[l + 1]
        xc = inputs.uniform(c.Nst, 100 + l)
        xf = inputs.uniform(f.Nst, 200 + l)
        out = torch.empty(f.Nst, dtype=dt, device="cuda")
        S.transfer(l, 0, _t(xc, dt), out)
        assert _rel(_np(out), mg.P[l] @ xc) < tol
        outc = torch.empty(c.Nst, dtype=dt, device="cuda")
        S.transfer(l, 1, _t(xf, dt), outc)
        assert _rel(_np(outc), mg.P[l].T @ xf) < tol
        outc.zero_()
        S.transfer(l, 2, _t(xf, dt), outc)
        nvc = (c.k + 1) * c.lay.Nv
        assert _rel(_np(outc)[:nvc], mg.I[l] @ xf[:(f.k + 1) * f.lay.Nv]) < tol


@pytest.mark.parametrize("d,n,r,k,amp,prec,keep", [(2, 8, 2, 2, 0.15, "fp64", 0), (2, 8, 1, 1, 0.0, "fp64", 0),
                                                   (2, 6, 1, 0, 0.1, "fp64", 0), (2, 8, 2, 2, 0.15, "fp32", 0),
                                                   (3, 4, 1, 1, 0.1, "fp32", 0),
                                                   # 3D Q3/P2: patches beyond shared memory (global path)
                                                   (3, 2, 2, 1, 0.1, "fp64", 0), (3, 4, 2, 1, 0.0, "fp32", 0),
                                                   # 3D Q4/P3: element tables and patches in global memory
                                                   (3, 2, 3, 1, 0.1, "fp64", 0), (3, 2, 3, 0, 0.0, "fp32", 0),
                                                   # p-coarsening in space only, DG(k) on every level
                                                   (2, 8, 2, 2, 0.15, "fp64", 1), (3, 4, 1, 2, 0.1, "fp32", 1)])
def test_smoother_and_vcycle_match_oracle(d, n, r, k, amp, prec, keep):
    """FP64: tight tolerances.  FP32 (the mixed-precision preconditioner): the error of each
    result against the FP64 oracle is bounded by 2e-3 relative (ill-conditioned patches)."""
    import torch
    S, mg, _ = _setup(d, n, r, k, amp, precision=prec, keep_time_degree=keep)
    assert [(L["n"], L["r"], L["k"]) for L in S.levels] == [(L.n, L.r, L.k) for L in mg.levels]
    dt = S.pdtype
    tol_s, tol_v, tol_x = (1e-9, 1e-11, 1e-13) if prec == "fp64" else (2e-3, 2e-3, 2e-6)
    L0 = mg.levels[0]
    U = inputs.uniform(L0.Nst, 7)
    mg.setup(U)
    S.smoother_build(_t(U))
    for l, L in enumerate(mg.levels):
        st = torch.empty(L.Nst, dtype=dt, device="cuda")
        S.level_state(l, st)
        nv = (L.k + 1) * L.lay.Nv
        assert _rel(_np(st)[:nv], mg.states[l][:nv]) < tol_x
    for l in range(len(mg.levels) - 1):
        L = mg.levels[l]
        rhs = inputs.uniform(L.Nst, 30 + l)
        d0 = inputs.uniform(L.Nst, 40 + l)
        want = mg.smoothers[l].sweep(mg.J[l], rhs, np.zeros(L.Nst))
        got = torch.empty(L.Nst, dtype=dt, device="cuda")
        S.smoother_sweep(l, _t(rhs, dt), got, 1, zero_start=True)
        assert _rel(_np(got), want) < tol_s, l
        want = mg.smoothers[l].sweep(mg.J[l], rhs, d0)
        got = _t(d0, dt)
        S.smoother_sweep(l, _t(rhs, dt), got, 1, zero_start=False)
        assert _rel(_np(got), want) < tol_s, l
    r0 = inputs.uniform(L0.Nst, 77)
    z = torch.empty(L0.Nst, dtype=torch.float64, device="cuda")
    S.vcycle(_t(r0), z)
    assert _rel(_np(z), mg.vcycle(r0)) < tol_v


@pytest.mark.parametrize("precision,d,n,r,k,amp,nu,tau,pname", [
    ("fp64", 2, 8, 1, 1, 0.0, 1e-2, 0.1, "TG2D"),   # 2D 8x8, Q2/P1, DG(1), dt = 0.1, Re = 100
    ("fp32", 2, 8, 1, 1, 0.0, 1e-2, 0.1, "TG2D"),
    ("fp64", 2, 8, 2, 2, 0.1, 1e-3, 0.05, "TG2D"),  # small case of the Q3/P2/DG(2) mapped workload
    ("fp32", 2, 8, 2, 2, 0.1, 1e-3, 0.05, "TG2D"),
    ("fp64", 2, 8, 1, 2, 0.1, 1e-2, 0.1, "MMS2D"),
    ("fp32", 2, 8, 1, 2, 0.1, 1e-2, 0.1, "MMS2D"),
    ("fp32", 3, 4, 1, 1, 0.1, 1.0 / 400, 0.05, "TG3D"),
    ("fp32", 3, 4, 1, 0, 0.0, 1e-2, 0.05, "MMS3D"),
    ("fp32", 3, 4, 1, 2, 0.1, 1.0 / 400, 0.01, "MMS3D"),   # small case of the 3D Q2/P1/DG(2) workload
    ("fp32", 3, 4, 2, 1, 0.0, 1.0 / 1600, 0.02, "TG3D"),   # small case of the 3D Q3/P2/DG(1) workload
    ("fp32", 3, 4, 2, 2, 0.0, 4e-4, 1.0 / 32, "CAV3D"),    # small case of the lid-driven cavity (Sec. 5.2)
    ("fp32", 3, 2, 3, 1, 0.1, 1.0 / 400, 0.05, "TG3D"),    # 3D Q4/P3 (global-memory element tables)
    ("fp32+keep", 2, 8, 2, 2, 0.1, 1e-3, 0.05, "TG2D"),    # p-coarsening in space only
])
def test_slab_solve_reaches_tolerance_and_matches_exact_solution(precision, d, n, r, k, amp, nu, tau, pname):
    import torch
    keep = int(precision.endswith("+keep"))
    S, mg, verts = _setup(d, n, r, k, amp, precision=precision.split("+")[0], nu=nu, tau=tau, problem=pname,
                          newton_rtol=1e-10, newton_atol=0.0, keep_time_degree=keep)
    L0 = mg.levels[0]
    prob = problems.make(pname, nu)
    V0 = torch.empty(L0.lay.Nv, dtype=torch.float64, device="cuda")
    S.initial_condition(V0)
    U = torch.empty(L0.Nst, dtype=torch.float64, device="cuda")
    S.initial_guess(V0, U)
    t0 = 0.2
    rc, st = S.slab_solve(t0, V0, U)
    assert rc == 0 and st["res_final"] <= 1e-10 * st["res0"]
    assert 1 <= st["newton_its"] <= 12 and st["rebuilds"] >= 1
    Vp = _np(V0)
    U0 = np.concatenate([np.tile(Vp, k + 1), np.zeros((k + 1) * L0.lay.Np)])
    Ud, _ = marching.newton_direct(L0.space, L0.td, U0, Vp, prob, t0, tol=1e-13)
    nv = (k + 1) * L0.lay.Nv
    got = _np(U)
    assert _rel(got[:nv], Ud[:nv]) < 1e-7
    # pressure: same up to the mean, which both remove
    assert np.abs(got[nv:] - Ud[nv:]).max() < 1e-6 * max(np.abs(Ud[nv:]).max(), 1.0)


@pytest.mark.parametrize("d,n,r,k,amp,prec", [(2, 8, 2, 2, 0.15, "fp64"), (2, 6, 1, 0, 0.1, "fp64"),
                                              (2, 8, 2, 2, 0.15, "fp32"), (3, 4, 1, 1, 0.1, "fp32")])
def test_fp16_patch_inverses(d, n, r, k, amp, prec):
    """Vanka sweeps with the patch inverses stored as FP16, one FP32 scale (the largest entry)
    per spatial inverse: every stored entry carries a relative error of at most 2^-11 of its
    block's largest entry; the sweep stays within 2e-2 relative of the FP64 oracle sweep."""
    import torch
    S, mg, _ = _setup(d, n, r, k, amp, precision=prec, vanka_fp16=1)
    dt = S.pdtype
    L0 = mg.levels[0]
    U = inputs.uniform(L0.Nst, 7)
    mg.setup(U)
    S.smoother_build(_t(U))
    for l in range(len(mg.levels) - 1):
        L = mg.levels[l]
        rhs = inputs.uniform(L.Nst, 30 + l)
        d0 = inputs.uniform(L.Nst, 40 + l)
        want = mg.smoothers[l].sweep(mg.J[l], rhs, d0)
        got = _t(d0, dt)
        S.smoother_sweep(l, _t(rhs, dt), got, 1, zero_start=False)
        assert _rel(_np(got), want) < 2e-2, l


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_slab_solve_with_fp16_patch_inverses(precision):
    """The FP16-stored smoother only changes the preconditioner: FGMRES still reaches the Newton
    tolerance and the solution equals the exact discrete solution (2D 8x8, Q3/P2, DG(2))."""
    import torch
    d, n, r, k, amp, nu, tau, pname = 2, 8, 2, 2, 0.1, 1e-3, 0.05, "TG2D"
    S, mg, verts = _setup(d, n, r, k, amp, precision=precision, nu=nu, tau=tau, problem=pname,
                          newton_rtol=1e-10, newton_atol=0.0, vanka_fp16=1)
    L0 = mg.levels[0]
    prob = problems.make(pname, nu)
    V0 = torch.empty(L0.lay.Nv, dtype=torch.float64, device="cuda")
    S.initial_condition(V0)
    U = torch.empty(L0.Nst, dtype=torch.float64, device="cuda")
    S.initial_guess(V0, U)
    rc, st = S.slab_solve(0.2, V0, U)
    assert rc == 0 and st["res_final"] <= 1e-10 * st["res0"]
    Vp = _np(V0)
    U0 = np.concatenate([np.tile(Vp, k + 1), np.zeros((k + 1) * L0.lay.Np)])
    Ud, _ = marching.newton_direct(L0.space, L0.td, U0, Vp, prob, 0.2, tol=1e-13)
    nv = (k + 1) * L0.lay.Nv
    got = _np(U)
    assert _rel(got[:nv], Ud[:nv]) < 1e-7
    assert np.abs(got[nv:] - Ud[nv:]).max() < 1e-6 * max(np.abs(Ud[nv:]).max(), 1.0)


@pytest.mark.parametrize("d,n,r,k,prec", [(2, 16, 2, 2, "fp32"), (3, 8, 1, 1, "fp64")])
def test_chunked_smoother_build_equals_single_chunk(d, n, r, k, prec):
    """The smoother build in chunks of cell planes (element matrices of a chunk plus one halo
    plane on either side) gives the same patch inverses, hence bit-identical sweeps, as one
    chunk over the whole level."""
    import torch
    from paper_2602_13841_gb300 import stmg
    build_and_load()
    verts = inputs.vertices(d, n, 0.1, 4)
    p0 = stmg.STMG_FP64 if prec == "fp64" else stmg.STMG_FP32
    out = []
    for chunk in (0, 2 * n ** (d - 1)):          # default (one chunk) / two planes per chunk
        p = stmg.default_params(dim=d, n_cells_1d=n, r=r, k=k, nu=1e-2, tau=0.05, problem="TG2D" if d == 2 else "TG3D",
                                precond_precision=p0, build_chunk_cells=chunk)
        S = stmg.Solver(p, verts)
        L = S.levels[0]
        S.smoother_build(_t(inputs.uniform(L["Nst"], 8)))
        got = _t(inputs.uniform(L["Nst"], 9), S.pdtype)
        S.smoother_sweep(0, _t(inputs.uniform(L["Nst"], 10), S.pdtype), got, 2, zero_start=False)
        torch.cuda.synchronize()
        out.append(got.cpu())
        S.close()
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("d,n,r,k,amp,prec", [(2, 8, 2, 2, 0.15, "fp64"), (2, 6, 1, 1, 0.0, "fp64"),
                                              (2, 7, 2, 0, 0.1, "fp32"), (3, 4, 1, 1, 0.1, "fp64"),
                                              (3, 4, 2, 1, 0.1, "fp32"), (3, 2, 3, 2, 0.1, "fp64")])
def test_diagonal_vanka_sweeps_match_oracle(d, n, r, k, amp, prec):
    """The diagonal space-time Vanka (smoother = 1): sweeps from zero and from a nonzero iterate on
    every smoothed level against the oracle's DiagonalVanka (FP64 1e-9, FP32 2e-3 relative)."""
    import torch
    from paper_2602_13841_gb300 import stmg
    build_and_load()
    verts = inputs.vertices(d, n, amp, 5)
    p = stmg.default_params(dim=d, n_cells_1d=n, r=r, k=k, nu=0.01, tau=0.05, problem="TG2D" if d == 2 else "TG3D",
                            precond_precision=stmg.STMG_FP64 if prec == "fp64" else stmg.STMG_FP32, smoother=1)
    S = stmg.Solver(p, verts)
    mg = multigrid.Multigrid(d, n, r, k, verts, 0.05, 0.01, smoother="diagonal")
    dt = S.pdtype
    tol = 1e-9 if prec == "fp64" else 2e-3
    U = inputs.uniform(mg.levels[0].Nst, 7)
    mg.setup(U)
    S.smoother_build(_t(U))
    for l in range(len(mg.levels) - 1):
        L = mg.levels[l]
        rhs = inputs.uniform(L.Nst, 30 + l)
        d0 = inputs.uniform(L.Nst, 40 + l)
        want = mg.smoothers[l].sweep(mg.J[l], rhs, np.zeros(L.Nst))
        got = torch.empty(L.Nst, dtype=dt, device="cuda")
        S.smoother_sweep(l, _t(rhs, dt), got, 1, zero_start=True)
        assert _rel(_np(got), want) < tol, l
        want = mg.smoothers[l].sweep(mg.J[l], rhs, d0)
        got = _t(d0, dt)
        S.smoother_sweep(l, _t(rhs, dt), got, 1, zero_start=False)
        assert _rel(_np(got), want) < tol, l


@pytest.mark.parametrize("precision,d,n,r,k,amp,nu,tau,pname", [
    ("fp32", 2, 8, 2, 2, 0.1, 1e-3, 0.05, "TG2D"),
    ("fp32", 3, 4, 2, 1, 0.0, 1.0 / 1600, 0.02, "TG3D"),
    ("fp32", 3, 2, 3, 1, 0.1, 1.0 / 400, 0.05, "TG3D"),   # 3D Q4/P3
])
def test_slab_solve_with_diagonal_vanka(precision, d, n, r, k, amp, nu, tau, pname):
    """The slab solve with the diagonal smoother reaches the Newton tolerance and the exact discrete
    solution (the smoother changes only the preconditioner)."""
    import torch
    S, mg, verts = _setup(d, n, r, k, amp, precision=precision, nu=nu, tau=tau, problem=pname,
                          newton_rtol=1e-10, newton_atol=0.0, smoother=1, nu1=2, nu2=2)
    L0 = mg.levels[0]
    prob = problems.make(pname, nu)
    V0 = torch.empty(L0.lay.Nv, dtype=torch.float64, device="cuda")
    S.initial_condition(V0)
    U = torch.empty(L0.Nst, dtype=torch.float64, device="cuda")
    S.initial_guess(V0, U)
    rc, st = S.slab_solve(0.2, V0, U)
    assert rc == 0 and st["res_final"] <= 1e-10 * st["res0"]
    Vp = _np(V0)
    U0 = np.concatenate([np.tile(Vp, k + 1), np.zeros((k + 1) * L0.lay.Np)])
    Ud, _ = marching.newton_direct(L0.space, L0.td, U0, Vp, prob, 0.2, tol=1e-13)
    nv = (k + 1) * L0.lay.Nv
    assert _rel(_np(U)[:nv], Ud[:nv]) < 1e-7


@pytest.mark.parametrize("d,n,r,k,amp,prec", [(2, 8, 2, 2, 0.15, "fp64"), (2, 6, 1, 1, 0.0, "fp32"),
                                              (3, 3, 1, 1, 0.1, "fp64")])
def test_exact_vanka_sweeps_match_oracle(d, n, r, k, amp, prec):
    """Exact space-time patches (smoother = 2; the convection of each time node at its own velocity):
    sweeps on every smoothed level against the oracle's ExactVanka (FP64 1e-9, FP32 2e-3)."""
    import torch
    from paper_2602_13841_gb300 import stmg
    build_and_load()
    verts = inputs.vertices(d, n, amp, 5)
    p = stmg.default_params(dim=d, n_cells_1d=n, r=r, k=k, nu=0.01, tau=0.05, problem="TG2D" if d == 2 else "TG3D",
                            precond_precision=stmg.STMG_FP64 if prec == "fp64" else stmg.STMG_FP32, smoother=2)
    S = stmg.Solver(p, verts)
    mg = multigrid.Multigrid(d, n, r, k, verts, 0.05, 0.01, smoother="exact")
    dt = S.pdtype
    tol = 1e-9 if prec == "fp64" else 2e-3
    U = inputs.uniform(mg.levels[0].Nst, 7)
    mg.setup(U)
    S.smoother_build(_t(U))
    for l in range(len(mg.levels) - 1):
        L = mg.levels[l]
        rhs = inputs.uniform(L.Nst, 30 + l)
        d0 = inputs.uniform(L.Nst, 40 + l)
        want = mg.smoothers[l].sweep(mg.J[l], rhs, d0)
        got = _t(d0, dt)
        S.smoother_sweep(l, _t(rhs, dt), got, 1, zero_start=False)
        assert _rel(_np(got), want) < tol, l


def test_slab_solve_with_exact_patches():
    """The slab solve with exact patches reaches the Newton tolerance and the exact solution."""
    import torch
    d, n, r, k, nu, tau = 2, 8, 2, 2, 1e-3, 0.05
    S, mg, verts = _setup(d, n, r, k, 0.1, precision="fp32", nu=nu, tau=tau, problem="TG2D",
                          newton_rtol=1e-10, newton_atol=0.0, smoother=2)
    L0 = mg.levels[0]
    prob = problems.make("TG2D", nu)
    V0 = torch.empty(L0.lay.Nv, dtype=torch.float64, device="cuda")
    S.initial_condition(V0)
    U = torch.empty(L0.Nst, dtype=torch.float64, device="cuda")
    S.initial_guess(V0, U)
    rc, st = S.slab_solve(0.2, V0, U)
    assert rc == 0 and st["res_final"] <= 1e-10 * st["res0"]
    Vp = _np(V0)
    U0 = np.concatenate([np.tile(Vp, k + 1), np.zeros((k + 1) * L0.lay.Np)])
    Ud, _ = marching.newton_direct(L0.space, L0.td, U0, Vp, prob, 0.2, tol=1e-13)
    nv = (k + 1) * L0.lay.Nv
    assert _rel(_np(U)[:nv], Ud[:nv]) < 1e-7
