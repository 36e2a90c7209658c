"""ILUTP (om_ilutp_factor): ILUT with threshold column pivoting, alone and
with equilibration, against the oracle (oracle.reorder_factor.ilutp, and
equilibrate for the scalings).

Bit-exact: the factor sizes, the number of swaps and the column permutation
q (both sides take every drop and pivot decision in FP64 from the same
elimination order).  Values: complex128 applications within 1e-10 of the
largest entry, complex64 within 1e-3 (the bounds of the unpivoted factors);
steady states within 1e-9 at eta <= 1e-12."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle.liouvillian import Params
from oracle.reorder_factor import equilibrate, ilutp
from oracle.steady import steady_state_dense
from paper_1411_4356_gb300 import api
from paper_1411_4356_gb300._lib import OMError
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)
FIG4 = dict(omega_m=1.0, Delta=-2.0, kappa=0.2, g0=0.5, E=0.1, Q_m=1e4)


def oparams(p):
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th, p.g2, p.lam)


def gpu_csr(M):
    rp, ci, va = M.export()
    return sp.csr_matrix((va, ci, rp), shape=(M.N, M.N))


CASES = [(3, 5, BASE, 1e-4, 10.0, 0.1), (4, 10, BASE, 1e-4, 10.0, 1.0),
         (4, 20, {**FIG4, "n_th": 0.0}, 1e-4, 100.0, 0.1), (4, 20, {**FIG4, "n_th": 1e-15}, 1e-4, 100.0, 0.1),
         (6, 20, BASE, 1e-5, 30.0, 0.5)]


@pytest.mark.parametrize("eq", [False, True])
@pytest.mark.parametrize("Nc,Nm,kw,d,fill,permtol", CASES)
def test_factor_and_apply_match_oracle(Nc, Nm, kw, d, fill, permtol, eq):
    p = SystemParams(Nc, Nm, **kw)
    A = api.build_liouvillian(p, "replace", nth_floor=0.0)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, d, fill, adjoint=True, fp64_sweeps=True, equilibrate=eq, permtol=permtol)
    B = gpu_csr(Ar)
    r = c = np.ones(Ar.N)
    if eq:
        r, c = equilibrate(B)
        B = sp.diags(r) @ B @ sp.diags(c)
    F = ilutp(B, d, fill, permtol)
    pivoted, swaps, q = api.ilu_pivots(M)
    assert pivoted and swaps == F.n_swaps
    np.testing.assert_array_equal(q, F.q)
    assert M.nnz_l == F.nnz_l and M.nnz_u == F.nnz_u
    rng = np.random.default_rng(Nc * 13 + Nm)
    v = rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)
    vt = torch.from_numpy(v).cuda()
    for h in (False, True):
        ref = r * F.solve_h(c * v) if h else c * F.solve(r * v)
        z = api.ilu_apply(M, vt, conj_transpose=h, fp64=True).cpu().numpy()
        np.testing.assert_allclose(z, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
        z32 = api.ilu_apply(M, vt, conj_transpose=h, fp64=False).cpu().numpy()
        assert np.abs(z32 - ref).max() <= 1e-3 * np.abs(ref).max()
    print(f"{Nc}x{Nm} permtol {permtol} eq {eq}: swaps {swaps}, fill {M.fill:.1f}")


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("eq", [False, True])
def test_solve_matches_dense_lu(precision, eq):
    p = SystemParams(4, 10, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, 1e-4, 10.0, equilibrate=eq, permtol=0.1)
    rho, info = api.steady_state_solve(Ar, M, perm, restart=30, tol=1e-13, precision=precision)
    assert info.eta <= 1e-12
    assert np.abs(rho.cpu().numpy() - steady_state_dense(oparams(p)).rho).max() <= 1e-9


def test_adjoint_solve_with_pivoted_factors():
    """The adjoint GMRES applies M^{-H} = diag(r) L^{-H} U^{-H} Q^T diag(c)."""
    from oracle.steady import adjoint_gradient_dense, observable_vec

    p = SystemParams(4, 10, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, 1e-4, 10.0, adjoint=True, equilibrate=True, permtol=0.1)
    rho, info = api.steady_state_solve(Ar, M, perm, restart=30, tol=1e-13)
    G = observable_vec(oparams(p), "n_b")
    G_t = torch.from_numpy(G.reshape((p.n, p.n), order="F")).cuda()
    g, ainfo = api.steady_state_adjoint(Ar, M, perm, rho, G_t, restart=30, tol=1e-13)
    ref = adjoint_gradient_dense(oparams(p), G)
    for t, name in enumerate(("Delta", "E", "g0", "kappa")):
        assert g[t] == pytest.approx(ref[name], rel=1e-8, abs=1e-12), name


def test_batched_engine_with_pivoted_factors():
    ps = [SystemParams(4, Nm, **{**BASE, "Delta": D}) for Nm, D in ((8, -1.0), (10, -0.5), (6, 0.3))]
    systems = []
    for p in ps:
        A = api.build_liouvillian(p)
        Ar, perm = api.permute(A)
        systems.append((Ar, api.ilu_factor(Ar, 1e-4, 10.0, equilibrate=True, permtol=0.1), perm))
    rhos, infos = api.steady_state_solve_batched(systems, restart=30, tol=1e-13)
    for p, rho, info in zip(ps, rhos, infos):
        assert info.status == 0 and info.eta <= 1e-12
        assert np.abs(rho.cpu().numpy() - steady_state_dense(oparams(p)).rho).max() <= 1e-9


def test_bad_permtol_is_rejected():
    p = SystemParams(3, 4, **BASE)
    Ar, perm = api.permute(api.build_liouvillian(p))
    for bad in (1.5, -0.1):
        with pytest.raises(OMError):
            api.ilu_factor(Ar, 1e-4, 10.0, permtol=bad)
    with pytest.raises(OMError):
        api.ilu_factor(Ar, 1e-4, 10.0, compensate=True, permtol=0.1)
