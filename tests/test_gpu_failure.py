"""Failure handling on the GPU without a GPU fault: the Vanka apply stages each patch inverse by
a bulk copy and waits for it on a shared-memory barrier with an iteration limit.  The test hook
stmg_test_wait_timeout makes that wait run out (the barrier expects bytes that are never sent);
the sweep must return STMG_ERR_TIMEOUT with its message, and once the hook is off the same handle
must give the sweep of a fresh handle again (the context stayed usable)."""
import ctypes

import numpy as np
import pytest

from tests.helpers import build_and_load, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


def _handle(r):
    import torch
    from paper_2602_13841_gb300 import inputs, stmg
    build_and_load()
    p = stmg.default_params(dim=2, n_cells_1d=4, r=r, k=1, nu=1e-2, tau=0.05, problem="TG2D",
                            precond_precision=stmg.STMG_FP32)
    S = stmg.Solver(p, inputs.vertices(2, 4, 0.1, 3))
    L = S.levels[0]
    S.smoother_build(torch.tensor(inputs.uniform(L["Nst"], 5), dtype=torch.float64, device="cuda"))
    return S


@pytest.mark.parametrize("r", [1, 2])     # one-warp patches (4 cells per block) / one cell per block
def test_vanka_wait_timeout_is_reported_and_the_handle_recovers(r):
    import torch
    from paper_2602_13841_gb300 import inputs, stmg
    S = _handle(r)
    L = S.levels[0]
    rhs = torch.tensor(inputs.uniform(L["Nst"], 11), dtype=torch.float32, device="cuda")
    d0 = torch.tensor(inputs.uniform(L["Nst"], 12), dtype=torch.float32, device="cuda")
    lib = S.lib
    assert lib.stmg_test_wait_timeout(S.h, 1) == 0
    d = d0.clone()
    st = lib.stmg_smoother_sweep(S.h, 0, ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(d.data_ptr()), 1, 0)
    assert st == 6, st                                  # STMG_ERR_TIMEOUT
    assert b"bounded wait" in lib.stmg_last_error(S.h)
    assert lib.stmg_test_wait_timeout(S.h, 0) == 0
    d = d0.clone()
    S.smoother_sweep(0, rhs, d, 1, zero_start=False)
    ref = _handle(r)
    d_ref = d0.clone()
    ref.smoother_sweep(0, rhs, d_ref, 1, zero_start=False)
    torch.cuda.synchronize()
    assert torch.equal(d, d_ref)
    assert float((d - d0).abs().max()) > 0.0


def test_noalloc_sweep_reports_the_wait_timeout_too():
    """The allocation-free sweep shares the Vanka apply and its bounded wait: with the hook on it
    must also return STMG_ERR_TIMEOUT, and the handle must recover afterwards."""
    import torch
    from paper_2602_13841_gb300 import inputs
    S = _handle(1)
    L = S.levels[0]
    lib = S.lib
    lib.stmg_smoother_sweep_noalloc.restype = ctypes.c_int
    lib.stmg_smoother_sweep_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_int, ctypes.c_int]
    rhs = torch.tensor(inputs.uniform(L["Nst"], 11), dtype=torch.float32, device="cuda")
    d0 = torch.tensor(inputs.uniform(L["Nst"], 12), dtype=torch.float32, device="cuda")
    assert lib.stmg_test_wait_timeout(S.h, 1) == 0
    d = d0.clone()
    st = lib.stmg_smoother_sweep_noalloc(S.h, 0, ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(d.data_ptr()), 1, 0)
    assert st == 6, st
    assert b"bounded wait" in lib.stmg_last_error(S.h)
    assert lib.stmg_test_wait_timeout(S.h, 0) == 0
    d = d0.clone()
    assert lib.stmg_smoother_sweep_noalloc(S.h, 0, ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                           1, 0) == 0
    d_ref = d0.clone()
    S.smoother_sweep(0, rhs, d_ref, 1, zero_start=False)
    torch.cuda.synchronize()
    assert torch.equal(d, d_ref)
