"""ILUT with the fill cap read as a running total, NNZ(L) + NNZ(U) <= p NNZ(A)
(om_ilu_factor flag 16), against the oracle's ILUT with cap="total": factor
sizes equal (a budget that binds and one that does not), applications within
the bounds of the per-row reading (complex128 1e-10, complex64 1e-3 of the
largest entry), steady states within 1e-9 of dense LU at eta <= 1e-12."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle.liouvillian import Params
from oracle.reorder_factor import ilut
from oracle.steady import steady_state_dense
from paper_1411_4356_gb300 import api
from paper_1411_4356_gb300._lib import OMError
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)
FIG4 = dict(omega_m=1.0, Delta=-1.0, kappa=0.2, g0=0.5, E=0.1, Q_m=1e4, n_th=3.0)


def oparams(p):
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th, p.g2, p.lam)


@pytest.mark.parametrize("Nc,Nm,kw,d,fill", [(3, 5, BASE, 1e-4, 1.5), (4, 10, BASE, 1e-4, 3.0), (4, 10, BASE, 1e-4, 100.0),
                                             (6, 20, BASE, 1e-5, 8.0), (4, 20, FIG4, 1e-4, 100.0)])
def test_factor_and_apply_match_oracle(Nc, Nm, kw, d, fill):
    p = SystemParams(Nc, Nm, **kw)
    A = api.build_liouvillian(p, "replace", nth_floor=0.0)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, d, fill, adjoint=True, fp64_sweeps=True, cap="total")
    rp, ci, va = Ar.export()
    F = ilut(sp.csr_matrix((va, ci, rp), shape=(Ar.N, Ar.N)), d, fill, cap="total")
    assert M.nnz_l == F.nnz_l and M.nnz_u == F.nnz_u
    assert M.nnz_l + M.nnz_u <= np.floor(fill * Ar.nnz) + Ar.N
    rng = np.random.default_rng(Nc * 17 + Nm)
    v = rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)
    vt = torch.from_numpy(v).cuda()
    for h in (False, True):
        ref = F.solve_h(v) if h else F.solve(v)
        z = api.ilu_apply(M, vt, conj_transpose=h, fp64=True).cpu().numpy()
        np.testing.assert_allclose(z, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
        z32 = api.ilu_apply(M, vt, conj_transpose=h, fp64=False).cpu().numpy()
        assert np.abs(z32 - ref).max() <= 1e-3 * np.abs(ref).max()
    print(f"{Nc}x{Nm} d {d} p {fill}: fill {M.fill:.2f}")


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_matches_dense_lu(precision):
    p = SystemParams(4, 10, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, 1e-4, 100.0, cap="total")
    rho, info = api.steady_state_solve(Ar, M, perm, restart=30, tol=1e-13, precision=precision)
    assert info.eta <= 1e-12
    assert np.abs(rho.cpu().numpy() - steady_state_dense(oparams(p)).rho).max() <= 1e-9


def test_total_budget_rejects_compensation():
    p = SystemParams(3, 4, **BASE)
    Ar, perm = api.permute(api.build_liouvillian(p))
    with pytest.raises(OMError):
        api.ilu_factor(Ar, 1e-4, 10.0, compensate=True, cap="total")
