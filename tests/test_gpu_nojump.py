"""The no-jump preconditioner S^{-1} (S: rho -> K rho + rho K^dag, the part of
Eq. 3 without the jump terms) and the steady states it leads to, through the
C ABI, against the oracle (oracle/nojump.py, oracle/steady.py).

Tolerances.  S^{-1} v is four products whose inputs are rounded to the
product precision u and accumulated in FP32: u = 2^-24 for the complex64
SIMT products, 2^-11 for TF32 on the tensor cores.  The eigenvector matrices
have condition numbers of about 20 on these systems, and each entry of a
product sums n terms, so the relative error of S^{-1} v (against its largest
entry) is of order kappa(V)^2 * u * sqrt(n): 5e-4 is allowed for complex64
and 5e-2 for TF32.  The steady states themselves come from FP64 flexible
GMRES on L~, so the precision of the preconditioner changes the iteration
count only: rho is held to the oracle within 1e-9 at eta <= 1e-13 (the same
bound as the ILU path)."""
import numpy as np
import pytest
import torch

from oracle.liouvillian import Params
from oracle.nojump import nojump_solve, steady_state_nojump
from oracle.steady import adjoint_gradient_dense, observable_vec, steady_state_dense
from paper_1411_4356_gb300 import api
from paper_1411_4356_gb300._lib import OMError
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)
APPLY_TOL = {False: 5e-4, True: 5e-2}  # keyed by tensor_cores


def oparams(p):
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th)


def rand_vec(N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(N) + 1j * rng.standard_normal(N)


@pytest.mark.parametrize("simt", [True, False])
@pytest.mark.parametrize("Nc,Nm", [(3, 5), (4, 10), (6, 20), (10, 20)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_apply_matches_oracle(Nc, Nm, adjoint, simt):
    p = SystemParams(Nc, Nm, 1.0, -1.0, 0.3, 0.5, 0.3, 1e4, 1.0)
    M = api.nojump_factor(p, adjoint=True, simt=simt)
    n = p.n
    v = rand_vec(n * n, Nc * 100 + Nm)
    z = api.nojump_apply(M, torch.from_numpy(v).cuda(), adjoint=adjoint).cpu().numpy()
    ref = nojump_solve(oparams(p), v, adjoint=adjoint)
    err = np.abs(z - ref).max() / np.abs(ref).max()
    print(f"{Nc}x{Nm} adjoint={adjoint} tc={M.tensor_cores} rel err {err:.2e} min|D| {M.min_abs_d:.3e}")
    assert err <= APPLY_TOL[M.tensor_cores]


@pytest.mark.parametrize("mode", ["replace", "add"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("simt", [True, False])
def test_solve_matches_dense_lu(mode, precision, simt):
    p = SystemParams(4, 10, **BASE)
    A = api.build_liouvillian(p, mode)
    M = api.nojump_factor(p, simt=simt)
    rho, info = api.steady_state_solve_nojump(A, M, restart=30, tol=1e-13, precision=precision)
    ref = steady_state_dense(oparams(p), mode).rho
    assert info.eta <= 1e-13
    assert np.abs(rho.cpu().numpy() - ref).max() <= 1e-9
    assert info.iterations <= 60


@pytest.mark.parametrize("Nc,Nm,kw", [(6, 20, dict(Delta=-1.3, kappa=0.4, g0=0.8, E=0.2, Q_m=1e3, n_th=0.2)),
                                      (10, 20, dict(Delta=-1.0, kappa=0.3, g0=0.5, E=0.3, Q_m=1e4, n_th=1.0)),
                                      (5, 24, dict(Delta=-0.5, kappa=0.5, g0=1.5, E=0.5, Q_m=1e4, n_th=0.0))])
def test_solve_matches_oracle(Nc, Nm, kw):
    """Larger systems against the oracle's own no-jump GMRES (FP64 Bartels-Stewart
    preconditioner), including n_th = 0 floored to 1e-15 (Sec. IV)."""
    p = SystemParams(Nc, Nm, omega_m=1.0, **kw)
    A = api.build_liouvillian(p)
    M = api.nojump_factor(p)
    rho, info = api.steady_state_solve_nojump(A, M, restart=50, tol=1e-14)
    x, its, ok, _ = steady_state_nojump(oparams(p), restart=50, rtol=1e-15)
    ref = x.reshape((p.n, p.n), order="F")
    err = np.abs(rho.cpu().numpy() - ref).max()
    print(f"{Nc}x{Nm}: its {info.iterations} (oracle {its}) eta {info.eta:.1e} err {err:.1e}")
    assert ok and info.eta <= 1e-14
    assert err <= 1e-9


def test_mixed_precision_matches_fp64():
    p = SystemParams(10, 20, 1.0, -1.0, 0.3, 0.5, 0.3, 1e4, 1.0)
    A = api.build_liouvillian(p)
    M = api.nojump_factor(p)
    r64, i64 = api.steady_state_solve_nojump(A, M, restart=50, tol=1e-14, precision=0)
    r32, i32 = api.steady_state_solve_nojump(A, M, restart=50, tol=1e-14, precision=1)
    assert i64.eta <= 1e-14 and i32.eta <= 1e-14
    assert np.abs(r64.cpu().numpy() - r32.cpu().numpy()).max() <= 1e-9


@pytest.mark.parametrize("mode", ["replace", "add"])
@pytest.mark.parametrize("which", ["n_a", "n_b"])
def test_adjoint_matches_oracle(mode, which):
    p = SystemParams(4, 10, **BASE)
    A = api.build_liouvillian(p, mode)
    M = api.nojump_factor(p, adjoint=True)
    rho, info = api.steady_state_solve_nojump(A, M, restart=30, tol=1e-13)
    G = observable_vec(oparams(p), which)
    g, ainfo = api.steady_state_adjoint_nojump(A, M, rho, torch.from_numpy(G).cuda().view(p.n, p.n).t(),
                                               restart=30, tol=1e-13)
    ref = adjoint_gradient_dense(oparams(p), G, mode)
    for t, name in enumerate(("Delta", "E", "g0", "kappa")):
        assert g[t] == pytest.approx(ref[name], rel=1e-8, abs=1e-12), name


def test_undamped_mode_is_rejected():
    """kappa = 0, n_th = 0 with no floor, g0 = E = 0: the states |c, 0> do not
    decay, lambda_i + conj(lambda_i) = 0 and S is singular."""
    p = SystemParams(3, 4, 1.0, -1.0, 0.0, 0.0, 0.0, 1e3, 0.0)
    with pytest.raises(OMError) as e:
        api.nojump_factor(p, nth_floor=0.0)
    assert e.value.status == -1


def test_single_level_is_rejected():
    """N_c = N_m = 1: L = 0 and S = 0, which has no inverse (the ILU path covers it)."""
    with pytest.raises(OMError):
        api.nojump_factor(SystemParams(1, 1, **BASE))


def test_permuted_matrix_is_rejected():
    p = SystemParams(3, 4, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.nojump_factor(p)
    with pytest.raises(OMError):
        api.steady_state_solve_nojump(Ar, M)


@pytest.mark.parametrize("Nc,Nm", [(1, 1), (1, 5), (2, 1), (3, 5), (4, 10), (6, 20)])
@pytest.mark.parametrize("mode", ["replace", "add"])
def test_stencil_operator_matches_oracle(Nc, Nm, mode):
    """y = L~ x from the stencil against the oracle's assembled L~ (Kronecker
    products) and against the library's CSR SpMV, including n_th = 0 floored."""
    from oracle.liouvillian import augmented

    for kw in (BASE, {**BASE, "n_th": 0.0}):
        p = SystemParams(Nc, Nm, **kw)
        A = api.build_liouvillian(p, mode)
        x = rand_vec(p.N, Nc * 7 + Nm)
        xt = torch.from_numpy(x).cuda()
        y = api.liouvillian_apply(A, xt).cpu().numpy()
        Lt, *_ = augmented(oparams(p), mode, 1e-15)
        ref = Lt @ x
        scale = np.abs(Lt).sum(axis=1).max() * np.abs(x).max()
        assert np.abs(y - ref).max() <= 1e-14 * scale
        assert np.abs(y - api.spmv(A, xt).cpu().numpy()).max() <= 1e-14 * scale
