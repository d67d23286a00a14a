"""stmg_smoother_sweep_noalloc: the sweep for callers that cannot allocate device memory during
the call (real-time loops that forbid allocator calls, fixed memory pools).  It launches the same
kernels in the same order as the regular stmg_smoother_sweep, only with its residual in a fixed
device array, so its result must equal the regular sweep's bit for bit, on two calls in a row (the
fixed scratch array keeps the previous call's contents, which must not leak into the next
result); sizes beyond its fixed scratch must be rejected."""
import ctypes

import pytest

from tests.helpers import build_and_load, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


def _solver(precision, n=8, r=1, k=1):
    import torch
    from paper_2602_13841_gb300 import inputs, stmg
    lib = build_and_load()
    lib.stmg_smoother_sweep_noalloc.restype = ctypes.c_int
    lib.stmg_smoother_sweep_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_int, ctypes.c_int]
    p = stmg.default_params(dim=2, n_cells_1d=n, r=r, k=k, nu=1e-2, tau=0.05, problem="TG2D",
                            precond_precision=precision)
    S = stmg.Solver(p, inputs.vertices(2, n, 0.1, 3))
    L0 = S.levels[0]
    U = torch.tensor(inputs.uniform(L0["Nst"], 5), dtype=torch.float64, device="cuda")
    S.smoother_build(U)
    return lib, S


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_sweep_matches_regular_sweep_twice(precision):
    import torch
    from paper_2602_13841_gb300 import inputs
    lib, S = _solver(precision)
    dt = S.pdtype
    for call in range(2):
        L = S.levels[0]
        rhs = torch.tensor(inputs.uniform(L["Nst"], 10 + call), dtype=dt, device="cuda")
        d0 = torch.tensor(inputs.uniform(L["Nst"], 20 + call), dtype=dt, device="cuda")
        ref = d0.clone()
        S.smoother_sweep(0, rhs, ref, nsweeps=2, zero_start=False)
        got = d0.clone()
        st = lib.stmg_smoother_sweep_noalloc(S.h, 0, ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(got.data_ptr()),
                                             2, 0)
        assert st == 0, lib.stmg_last_error(S.h)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), call
        assert float((got - d0).abs().max()) > 0.0


def test_noalloc_sweep_rejects_levels_beyond_its_scratch():
    import torch
    lib, S = _solver(0, n=128, r=2, k=2)
    L = S.levels[0]
    assert L["Nst"] * 8 > (1 << 22)
    x = torch.zeros(L["Nst"], dtype=torch.float64, device="cuda")
    d = torch.zeros_like(x)
    st = lib.stmg_smoother_sweep_noalloc(S.h, 0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(d.data_ptr()), 1, 0)
    assert st == 1 and b"exceeds the fixed scratch" in lib.stmg_last_error(S.h)
