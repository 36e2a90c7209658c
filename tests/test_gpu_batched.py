"""Batched solves (om_steady_state_solve_batched): systems of uneven size and
detuning solved together must each match the oracle, and the lock-step and
stream-per-solve engines must agree with one-by-one solves."""
import numpy as np
import pytest

from oracle.liouvillian import Params
from oracle.steady import steady_state_dense
from paper_1411_4356_gb300 import api
from paper_1411_4356_gb300.workloads import SystemParams, batched_draws

pytestmark = pytest.mark.gpu


def oparams(p):
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th)


def prepare(p, d=1e-4, fill=20.0):
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, d, fill)
    return Ar, M, perm


def uneven_params():
    rng = np.random.default_rng(4356)
    return [SystemParams(4, int(nm), 1.0, float(dl), 0.4, 0.8, 0.2, 1e3, 0.2)
            for dl, nm in zip(rng.uniform(-3, 1, 9), rng.choice([6, 8, 10], 9))]


@pytest.mark.parametrize("concurrency", [0, 4])
def test_batched_uneven_sizes_match_dense(concurrency):
    params = uneven_params()
    systems = [prepare(p) for p in params]
    rhos, infos = api.steady_state_solve_batched(systems, restart=30, tol=1e-12, concurrency=concurrency)
    for p, rho, info in zip(params, rhos, infos):
        assert info.status == 0 and info.eta <= 1e-12
        ref = steady_state_dense(oparams(p)).rho
        assert np.abs(rho.cpu().numpy() - ref).max() <= 1e-9


def test_lockstep_tail_systems_retire():
    """A batch whose members need very different iteration counts (one with
    restart cycles, one converging in a few steps) retires each on its own."""
    params = [SystemParams(3, 4, 1.0, -1.0, 0.4, 0.5, 0.2, 1e3, 0.2),
              SystemParams(4, 10, 1.0, -1.0, 0.4, 0.8, 0.2, 1e3, 0.2)]
    systems = [prepare(params[0], 0.0, 100.0), prepare(params[1], 1e-3, 10.0)]
    rhos, infos = api.steady_state_solve_batched(systems, restart=8, tol=1e-12)
    assert infos[0].iterations < infos[1].iterations
    assert infos[1].cycles > 1
    for p, rho, info in zip(params, rhos, infos):
        assert info.status == 0 and info.eta <= 1e-12
        ref = steady_state_dense(oparams(p)).rho
        assert np.abs(rho.cpu().numpy() - ref).max() <= 1e-9


def test_lockstep_rejects_other_precisions():
    systems = [prepare(uneven_params()[0])]
    with pytest.raises(RuntimeError, match="lock-step"):
        api.steady_state_solve_batched(systems, precision=1)


@pytest.mark.parametrize("concurrency", [0, 2])
def test_batched_equals_single_solves_on_sweep_draws(concurrency):
    """The first draws of the 512-system sweep (N_c = 6, N_m in {20..60}).
    The stream engine runs the single-solve kernels on the same inputs (equal
    iteration counts); the lock-step engine reduces in another order, so its
    counts may differ by a step at the stopping test."""
    params = batched_draws(4)
    systems = [prepare(p, 1e-5, 60.0) for p in params]
    rhos, infos = api.steady_state_solve_batched(systems, restart=30, tol=1e-11, concurrency=concurrency)
    for (Ar, M, perm), rho, info in zip(systems, rhos, infos):
        assert info.status == 0 and info.eta <= 1e-11
        single, sinfo = api.steady_state_solve(Ar, M, perm, restart=30, tol=1e-11)
        if concurrency:
            assert sinfo.iterations == info.iterations
            assert float((single - rho).abs().max()) <= 1e-12
        else:
            assert abs(sinfo.iterations - info.iterations) <= 2
            assert float((single - rho).abs().max()) <= 1e-9
