"""The no-jump parameter sweep (om_steady_state_sweep_nojump): many systems,
each through the whole path on concurrent streams, against dense LU (the
oracle) and against the same systems solved one by one; a failing system
does not stop the others; the result does not depend on the concurrency.
Tolerances: rho within 1e-9 of dense LU at eta <= 1e-12 (as for single
solves); the sweep and the one-by-one solves run the same kernels in the same
order and agree to 1e-12."""
import numpy as np
import pytest

from oracle.liouvillian import Params
from oracle.steady import steady_state_dense
from paper_1411_4356_gb300 import api
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, kappa=0.4, g0=0.8, E=0.2, Q_m=1e3, n_th=0.2)


def oparams(p):
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th, p.g2, p.lam)


def draws(count, seed=7):
    rng = np.random.default_rng(seed)
    return [SystemParams(int(rng.integers(3, 6)), int(rng.choice([6, 8, 10, 12])), Delta=float(rng.uniform(-3, 1)),
                         **BASE) for _ in range(count)]


@pytest.mark.parametrize("concurrency", [1, 4])
def test_sweep_matches_dense_lu(concurrency):
    ps = draws(10)
    rhos, infos = api.steady_state_sweep_nojump(ps, restart=40, tol=1e-13, concurrency=concurrency)
    for p, rho, info in zip(ps, rhos, infos):
        assert info.status == 0 and info.eta <= 1e-12
        ref = steady_state_dense(oparams(p)).rho
        assert np.abs(rho.cpu().numpy() - ref).max() <= 1e-9


def test_sweep_equals_one_by_one_solves():
    ps = draws(6, seed=11)
    rhos, infos = api.steady_state_sweep_nojump(ps, restart=40, tol=1e-13, precision=1, concurrency=3)
    for p, rho, info in zip(ps, rhos, infos):
        A = api.build_liouvillian(p)
        M = api.nojump_factor(p)
        r1, i1 = api.steady_state_solve_nojump(A, M, restart=40, tol=1e-13, precision=1)
        assert info.iterations == i1.iterations
        assert (rho - r1).abs().max().item() <= 1e-12


def test_failing_system_does_not_stop_the_others():
    """An undamped system (kappa = g0 = E = n_th = 0, no floor) has no no-jump
    inverse; its status is OM_EINVAL and the other systems are solved."""
    ps = draws(4, seed=3)
    ps.insert(2, SystemParams(3, 4, 1.0, -1.0, 0.0, 0.0, 0.0, 1e3, 0.0))
    rhos, infos = api.steady_state_sweep_nojump(ps, restart=40, tol=1e-13, nth_floor=0.0, concurrency=2)
    assert infos[2].status == -1
    for k in (0, 1, 3, 4):
        assert infos[k].status == 0
        ref = steady_state_dense(oparams(ps[k]), nth_floor=0.0).rho
        assert np.abs(rhos[k].cpu().numpy() - ref).max() <= 1e-9


def test_empty_sweep():
    rhos, infos = api.steady_state_sweep_nojump([], concurrency=2)
    assert rhos == [] and infos == []
