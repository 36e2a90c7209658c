"""om_set_allocator: every device allocation of the library goes through the
hook -- here PyTorch's caching allocator -- and is returned through it."""
import gc

import numpy as np
import pytest
import torch

from paper_1411_4356_gb300 import api
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


def test_handles_and_solves_allocate_through_the_hook():
    gc.collect()  # tensors of earlier tests still waiting for collection
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    calls0 = api.allocator_hook_calls()
    api.use_torch_allocator(True)
    try:
        p = SystemParams(6, 20, **BASE)
        A = api.build_liouvillian(p)
        M = api.nojump_factor(p, adjoint=True)
        held = torch.cuda.memory_allocated() - base
        assert held >= A.nnz * 16  # the CSR values alone
        rho, info = api.steady_state_solve_nojump(A, M, tol=1e-12, precision=1)
        Ar, perm = api.permute(A)
        F = api.ilu_factor(Ar, 1e-4, 20.0)
        rho2, info2 = api.steady_state_solve(Ar, F, perm, tol=1e-12)
        assert np.abs(rho.cpu().numpy() - rho2.cpu().numpy()).max() <= 1e-9
        assert api.allocator_hook_calls() - calls0 > 20
        for h in (F, Ar, M, A):
            h.free()
        del rho, rho2, perm
        torch.cuda.synchronize()
        gc.collect()
        assert torch.cuda.memory_allocated() <= base
    finally:
        api.use_torch_allocator(False)


def test_default_allocator_restored():
    api.use_torch_allocator(False)
    calls0 = api.allocator_hook_calls()
    p = SystemParams(3, 4, **BASE)
    A = api.build_liouvillian(p)
    A.free()
    assert api.allocator_hook_calls() == calls0
