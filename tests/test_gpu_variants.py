"""The Hamiltonian variants of Sec. VI through the whole CUDA path: the
quadratic coupling g2 (b + b^dag)^2 a^dag a and the anharmonic term
lam (b + b^dag)^4, each added to Eq. 1 (oracle/liouvillian.py holds the
definition and its pins).

Checked against the oracle: the assembled L~ (structure bit-exact, values
within 16 eps ||L||_inf as for Eq. 1 alone), the stencil operator, the
effective Hamiltonian inside the no-jump preconditioner, and the steady states
of both preconditioned paths (RCM + ILUT and no-jump) against dense LU, within
1e-9 at eta <= 1e-12.  Cutoffs N_m <= 4 leave the X^4 bands (and for N_m <= 2
the X^2 bands) empty: those sizes are in the parameter lists."""
import numpy as np
import pytest
import torch

from oracle.liouvillian import Params, augmented
from oracle.nojump import nojump_solve
from oracle.steady import steady_state_dense
from paper_1411_4356_gb300 import api
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)
# g2 and lam are chosen so that no band entry g2 c (X^2)_{m,m+2} + lam (X^4)_{m,m+2}
# cancels exactly (an exact zero would be dropped on one side only by rounding)
VARIANTS = [dict(g2=0.05), dict(lam=0.004), dict(g2=-0.03, lam=0.00217), dict(g0=0.0, g2=0.08)]


def oparams(p):
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th, p.g2, p.lam)


def assembly_atol(L):
    return 16 * np.finfo(float).eps * max(float(np.abs(L).sum(axis=1).max()), 1e-300)


@pytest.mark.parametrize("kw", VARIANTS)
@pytest.mark.parametrize("Nc,Nm", [(1, 1), (2, 2), (2, 3), (3, 4), (2, 5), (3, 9), (4, 12)])
@pytest.mark.parametrize("mode", ["replace", "add"])
def test_assembly_matches_oracle(kw, Nc, Nm, mode):
    p = SystemParams(Nc, Nm, **{**BASE, **kw})
    A = api.build_liouvillian(p, mode)
    Lt, b, w, L = augmented(oparams(p), mode, 1e-15)
    rp, ci, va = A.export()
    np.testing.assert_array_equal(rp, Lt.indptr)
    np.testing.assert_array_equal(ci, Lt.indices)
    assert np.abs(va - Lt.data).max(initial=0.0) <= assembly_atol(L)
    assert A.w == pytest.approx(w, rel=1e-13)
    assert A.norm_inf == pytest.approx(np.abs(L).sum(axis=1).max(), rel=1e-14)


@pytest.mark.parametrize("kw", VARIANTS)
@pytest.mark.parametrize("Nc,Nm", [(2, 3), (3, 9), (4, 12)])
@pytest.mark.parametrize("mode", ["replace", "add"])
def test_stencil_matches_oracle(kw, Nc, Nm, mode):
    p = SystemParams(Nc, Nm, **{**BASE, **kw})
    A = api.build_liouvillian(p, mode)
    rng = np.random.default_rng(Nc * 31 + Nm)
    x = rng.standard_normal(p.N) + 1j * rng.standard_normal(p.N)
    xt = torch.from_numpy(x).cuda()
    y = api.liouvillian_apply(A, xt).cpu().numpy()
    Lt, *_ = augmented(oparams(p), mode, 1e-15)
    ref = Lt @ x
    scale = np.abs(Lt).sum(axis=1).max() * np.abs(x).max()
    assert np.abs(y - ref).max() <= 1e-14 * scale
    assert np.abs(y - api.spmv(A, xt).cpu().numpy()).max() <= 1e-14 * scale


@pytest.mark.parametrize("kw", VARIANTS)
def test_nojump_apply_matches_oracle(kw):
    """S^{-1} with K = -i H - (1/2) sum gamma O^dag O built from the variant H;
    complex64 SIMT products (relative 5e-4, the bound of the Eq. 1 tests)."""
    p = SystemParams(3, 10, **{**BASE, **kw})
    M = api.nojump_factor(p, simt=True)
    rng = np.random.default_rng(17)
    v = rng.standard_normal(p.N) + 1j * rng.standard_normal(p.N)
    z = api.nojump_apply(M, torch.from_numpy(v).cuda()).cpu().numpy()
    ref = nojump_solve(oparams(p), v)
    assert np.abs(z - ref).max() / np.abs(ref).max() <= 5e-4


@pytest.mark.parametrize("kw", VARIANTS)
@pytest.mark.parametrize("path", ["ilu", "nojump"])
def test_steady_state_matches_dense_lu(kw, path):
    p = SystemParams(4, 12, **{**BASE, **kw})
    ref = steady_state_dense(oparams(p), "replace").rho
    A = api.build_liouvillian(p)
    if path == "ilu":
        Ar, perm = api.permute(A)
        M = api.ilu_factor(Ar, 1e-6, 40.0)
        rho, info = api.steady_state_solve(Ar, M, perm, restart=30, tol=1e-13)
    else:
        M = api.nojump_factor(p)
        rho, info = api.steady_state_solve_nojump(A, M, restart=40, tol=1e-13)
    assert info.eta <= 1e-12
    assert np.abs(rho.cpu().numpy() - ref).max() <= 1e-9


def test_variants_change_the_state():
    """A nonzero g2 or lam moves the steady state (the terms are not dropped)."""
    p0 = SystemParams(3, 12, **BASE)
    A0 = api.build_liouvillian(p0)
    r0, _ = api.steady_state_solve_nojump(A0, api.nojump_factor(p0), restart=40, tol=1e-13)
    for kw in VARIANTS[:2]:
        p = p0.with_(**kw)
        A = api.build_liouvillian(p)
        r, _ = api.steady_state_solve_nojump(A, api.nojump_factor(p), restart=40, tol=1e-13)
        assert (r - r0).abs().max().item() > 1e-6
