"""Equilibrated ILUT (om_ilu_factor flag 8): the factors of diag(r) A diag(c)
with r = 1 / row maxima and c = 1 / column maxima of diag(r) A, applied as
M^{-1} = diag(c) (L U)^{-1} diag(r) and M^{-H} = diag(r) (L U)^{-H} diag(c),
against the oracle (oracle.reorder_factor.equilibrate and ilut).

Tolerances as for the unscaled factors (tests/test_gpu_parity.py): factor
sizes bit-exact, complex128 applications within 1e-10 of the largest entry,
complex64 within 1e-3, the condition estimate within 1e-10 (FP64) relative,
steady states within 1e-9 at eta <= 1e-12."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle.liouvillian import Params
from oracle.reorder_factor import equilibrate, ilut
from oracle.steady import steady_state_dense, steady_state_iterative
from paper_1411_4356_gb300 import api
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


def oparams(p):
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th, p.g2, p.lam)


def gpu_csr(M):
    rp, ci, va = M.export()
    return sp.csr_matrix((va, ci, rp), shape=(M.N, M.N))


@pytest.mark.parametrize("Nc,Nm,d,fill", [(3, 5, 1e-4, 10.0), (4, 10, 1e-4, 10.0), (6, 20, 1e-5, 30.0)])
def test_apply_matches_oracle(Nc, Nm, d, fill):
    p = SystemParams(Nc, Nm, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, d, fill, adjoint=True, fp64_sweeps=True, equilibrate=True)
    B = gpu_csr(Ar)
    r, c = equilibrate(B)
    F = ilut(sp.diags(r) @ B @ sp.diags(c), d, fill)
    assert M.nnz_l == F.nnz_l and M.nnz_u == F.nnz_u
    rng = np.random.default_rng(11)
    v = rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)
    vt = torch.from_numpy(v).cuda()
    for h in (False, True):
        ref = r * F.solve_h(c * v) if h else c * F.solve(r * v)
        z = api.ilu_apply(M, vt, conj_transpose=h, fp64=True).cpu().numpy()
        np.testing.assert_allclose(z, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
        z32 = api.ilu_apply(M, vt, conj_transpose=h, fp64=False).cpu().numpy()
        assert np.abs(z32 - ref).max() <= 1e-3 * np.abs(ref).max()
    ce = np.abs(c * F.solve(r * np.ones(Ar.N, dtype=complex))).max()
    assert abs(api.ilu_condest(M, fp64=True) - ce) <= 1e-10 * ce


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mode", ["replace", "add"])
def test_solve_matches_dense_lu(precision, mode):
    p = SystemParams(4, 10, **BASE)
    A = api.build_liouvillian(p, mode)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, 1e-4, 10.0, equilibrate=True)
    rho, info = api.steady_state_solve(Ar, M, perm, restart=30, tol=1e-13, precision=precision)
    ref = steady_state_dense(oparams(p), mode).rho
    assert info.eta <= 1e-12
    assert np.abs(rho.cpu().numpy() - ref).max() <= 1e-9


def test_solve_matches_oracle_iterative():
    """The oracle's own equilibrated pipeline (RCM, scaling, ILUT, GMRES) at 6x20."""
    p = SystemParams(6, 20, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, 1e-5, 30.0, equilibrate=True)
    rho, info = api.steady_state_solve(Ar, M, perm, restart=30, tol=1e-13)
    ref = steady_state_iterative(oparams(p), droptol=1e-5, fill=30.0, restart=30, rtol=1e-14,
                                 equilibrated=True)
    assert ref.converged and info.eta <= 1e-12
    assert np.abs(rho.cpu().numpy() - ref.rho).max() <= 1e-9


def test_batched_engine_applies_the_scalings():
    ps = [SystemParams(4, Nm, **{**BASE, "Delta": D}) for Nm, D in ((8, -1.0), (10, -0.5), (6, 0.3))]
    systems = []
    for p in ps:
        A = api.build_liouvillian(p)
        Ar, perm = api.permute(A)
        systems.append((Ar, api.ilu_factor(Ar, 1e-4, 10.0, equilibrate=True), perm))
    rhos, infos = api.steady_state_solve_batched(systems, restart=30, tol=1e-13)
    for p, rho, info in zip(ps, rhos, infos):
        assert info.status == 0 and info.eta <= 1e-12
        ref = steady_state_dense(oparams(p)).rho
        assert np.abs(rho.cpu().numpy() - ref).max() <= 1e-9
