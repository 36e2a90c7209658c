"""Device-side waits that run out: a solve given wait_timeout_ns = 1 ns has
every spin-wait of its kernels (the mbarrier phases of the tensor-core
products and of the triangular sweeps, the split sweep's cross-block flags)
give up at once.  The kernels abort -- draining their own copies in flight and
freeing their tensor memory -- and the solve returns OM_ETIMEOUT, distinct
from OM_ENUMERIC.  No GPU fault is involved; the same handles then solve
normally."""
import numpy as np
import pytest

from paper_1411_4356_gb300 import api
from paper_1411_4356_gb300._lib import OMError
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)
ETIMEOUT = -8


@pytest.mark.parametrize("precision", [0, 1])
def test_no_jump_products_time_out(precision):
    p = SystemParams(6, 20, **BASE)
    A = api.build_liouvillian(p)
    M = api.nojump_factor(p)
    assert M.tensor_cores
    with pytest.raises(OMError) as e:
        api.steady_state_solve_nojump(A, M, tol=1e-12, precision=precision, max_iters=200, wait_timeout_ns=1)
    assert e.value.status == ETIMEOUT, e.value
    rho, info = api.steady_state_solve_nojump(A, M, tol=1e-12, precision=precision)
    assert info.status == 0 and info.eta <= 1e-12


@pytest.mark.parametrize("fp64_sweeps", [False, True])
def test_ilu_sweeps_time_out(fp64_sweeps):
    """complex64 sweeps run split over all SMs; complex128 sweeps in one block.
    A wait whose phase is already complete at its first poll (mbarrier
    try_wait itself waits a little) succeeds even with a 1 ns limit, so a
    one-block sweep whose copies all land in time can finish: the solve is
    tried a few times, each attempt must end in OM_ETIMEOUT or succeed, and
    at least one must time out."""
    p = SystemParams(10, 20, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, 1e-4, 20.0, fp64_sweeps=fp64_sweeps)
    api.profile(True)
    statuses = []
    for _ in range(5):
        try:
            api.steady_state_solve(Ar, M, perm, tol=1e-12, max_iters=200, wait_timeout_ns=1,
                                   precond_fp64=fp64_sweeps)
            statuses.append(0)
        except OMError as e:
            statuses.append(e.status)
        if ETIMEOUT in statuses:
            break
    _, nsplit = api.profile_read(api.PROF_SPLIT)
    _, nblock = api.profile_read(api.PROF_SWEEP)
    api.profile(False)
    assert set(statuses) <= {0, ETIMEOUT} and ETIMEOUT in statuses, statuses
    assert (nsplit > 0) != fp64_sweeps and (nblock > 0) == fp64_sweeps
    rho, info = api.steady_state_solve(Ar, M, perm, tol=1e-12, precond_fp64=fp64_sweeps)
    assert info.status == 0 and np.isfinite(rho.abs().max().item())
