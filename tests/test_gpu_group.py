"""Batched preconditioning across same-shape solves (stmg_group_*): handles of one shape attached to
a group run their V-cycles as batched launches (one launch per kernel for all ready slots).  Each
slot computes what a handle without a group computes, so every solve -- run concurrently with the
others on its own host thread and stream -- must give the same bits as the same request solved
alone without a group; and the batching must actually happen (fewer rounds than V-cycles)."""
import threading

import numpy as np
import pytest

from tests.helpers import build_and_load, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]

CASES = [(2, 8, 2, 2, "TG2D", 0.1), (2, 6, 1, 1, "MMS2D", 0.0), (3, 4, 1, 1, "TG3D", 0.1)]


def _solve(S, V0, U, t0):
    S.initial_guess(V0, U)
    rc, st = S.slab_solve(t0, V0, U, check=False)
    return rc, st


@pytest.mark.parametrize("d,n,r,k,pname,amp", CASES)
def test_group_solves_equal_solo_solves_bitwise(d, n, r, k, pname, amp):
    import torch
    from paper_2602_13841_gb300 import inputs, stmg
    build_and_load()
    verts = inputs.vertices(d, n, amp, 3)
    res = [1.0 / 100, 1.0 / 700, 1.0 / 1500]

    def params(nu):
        return stmg.default_params(dim=d, n_cells_1d=n, r=r, k=k, nu=nu, tau=0.05, problem=pname,
                                   precond_precision=stmg.STMG_FP32, newton_rtol=1e-10, newton_atol=1e-14,
                                   nu1=2, nu2=2)

    def run(S, out, i):
        with torch.cuda.stream(torch.cuda.ExternalStream(S.stream)):
            L = S.levels[0]
            V0 = torch.empty(L["Nv"], dtype=torch.float64, device="cuda")
            U = torch.empty(L["Nst"], dtype=torch.float64, device="cuda")
            S.initial_condition(V0)
            rc, st = _solve(S, V0, U, 0.1)
            torch.cuda.current_stream().synchronize()
            out[i] = (rc, st, U.cpu().numpy())

    # alone, without a group
    solo = {}
    for i, nu in enumerate(res):
        S = stmg.Solver(params(nu), verts, stream=torch.cuda.Stream().cuda_stream)
        run(S, solo, i)
        S.close()
    # the same three requests at once, attached to one group
    G = stmg.Group(params(res[0]), verts, slots=3)
    solvers = [stmg.Solver(params(nu), verts, stream=torch.cuda.Stream().cuda_stream) for nu in res]
    for S in solvers:
        G.attach(S)
    mixed = {}
    threads = [threading.Thread(target=run, args=(S, mixed, i)) for i, S in enumerate(solvers)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    stats = G.stats()
    for S in solvers:
        G.detach(S)
        S.close()
    G.close()
    for i in range(len(res)):
        assert solo[i][0] == 0 and mixed[i][0] == 0, (solo[i][1], mixed[i][1])
        assert solo[i][1]["gmres_its_total"] == mixed[i][1]["gmres_its_total"]
        assert np.array_equal(solo[i][2], mixed[i][2]), i
    # batching happened: every FGMRES iteration asked for one slot V-cycle, rounds served several
    assert stats["slot_vcycles"] == sum(m[1]["gmres_its_total"] for m in mixed.values())
    assert stats["rounds"] < stats["slot_vcycles"]


def test_group_rejects_a_different_shape():
    import torch
    from paper_2602_13841_gb300 import inputs, stmg
    build_and_load()
    p = stmg.default_params(dim=2, n_cells_1d=8, r=1, k=1, nu=0.01, tau=0.05, problem="TG2D")
    q = stmg.default_params(dim=2, n_cells_1d=8, r=2, k=1, nu=0.01, tau=0.05, problem="TG2D")
    G = stmg.Group(p, inputs.vertices(2, 8, 0.0, 1), slots=2)
    S = stmg.Solver(q, inputs.vertices(2, 8, 0.0, 1))
    with pytest.raises(stmg.StmgError):
        G.attach(S)
    S.close()
    G.close()
