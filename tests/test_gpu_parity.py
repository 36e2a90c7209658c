"""Parity of the CUDA path (through the C ABI) with the oracle.

Tolerances: integer and index data (row pointers, columns, the RCM
permutation) bit-exact; assembled values within 16 eps ||L||_inf (the oracle
sums up to eight Kronecker terms per entry, each rounded at the size of its
own terms -- |H_ii| can be far larger than the difference H_ii - H_jj it
feeds -- while the stencil forms each entry directly); vectors within
1e-13 / 1e-10 relative to their maximum; rho within 1e-9 absolute at
eta <= 1e-10 (the target the method is held to)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle.liouvillian import Params, augmented, liouvillian
from oracle.reorder_factor import ilut, permute_symmetric, rcm_permutation
from oracle.steady import eta as oracle_eta, observables, steady_state_dense, steady_state_iterative
from paper_1411_4356_gb300 import TINY, api
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


def oparams(p: SystemParams) -> Params:
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th)


def assembly_atol(L):
    return 16 * np.finfo(float).eps * max(float(np.abs(L).sum(axis=1).max()), 1e-300)


def gpu_csr(M):
    rp, ci, va = M.export()
    return sp.csr_matrix((va, ci, rp), shape=(M.N, M.N))


# ------------------------------------------------------------------ assembly
@pytest.mark.parametrize("Nc,Nm", [(1, 1), (1, 5), (2, 1), (3, 5), (4, 8), (4, 10), (6, 20)])
@pytest.mark.parametrize("mode", ["replace", "add"])
def test_assembly_matches_oracle(Nc, Nm, mode):
    p = SystemParams(Nc, Nm, **BASE)
    A = api.build_liouvillian(p, mode)
    Lt, b, w, L = augmented(oparams(p), mode, 1e-15)
    rp, ci, va = A.export()
    np.testing.assert_array_equal(rp, Lt.indptr)
    np.testing.assert_array_equal(ci, Lt.indices)
    assert np.abs(va - Lt.data).max(initial=0.0) <= assembly_atol(L)
    assert A.w == pytest.approx(w, rel=1e-13)
    Linf = np.abs(L).sum(axis=1).max()
    assert A.norm_inf == pytest.approx(Linf, rel=1e-14)


def test_assembly_zero_temperature_and_parameters_zero():
    for kw in [dict(n_th=0.0), dict(g0=0.0), dict(E=0.0), dict(kappa=0.0)]:
        p = SystemParams(3, 6, **{**BASE, **kw})
        for floor in (0.0, 1e-15):
            A = api.build_liouvillian(p, "replace", floor)
            Lt, _, _, L = augmented(oparams(p), "replace", floor)
            rp, ci, va = A.export()
            np.testing.assert_array_equal(rp, Lt.indptr)
            np.testing.assert_array_equal(ci, Lt.indices)
            assert np.abs(va - Lt.data).max(initial=0.0) <= assembly_atol(L)


def test_fig1_nnz_on_gpu():
    A = api.build_liouvillian(SystemParams(4, 8, **BASE), "add")
    assert A.nnz == 8957


# ------------------------------------------------------------------ RCM
@pytest.mark.parametrize("Nc,Nm", [(2, 3), (3, 5), (4, 8), (4, 10), (6, 20), (10, 20)])
@pytest.mark.parametrize("mode", ["replace", "add"])
def test_permutation_bit_exact(Nc, Nm, mode):
    p = SystemParams(Nc, Nm, **BASE)
    A = api.build_liouvillian(p, mode)
    Ar, perm = api.permute(A)
    Lt, _, _, L = augmented(oparams(p), mode, 1e-15)
    ref = rcm_permutation(Lt)
    np.testing.assert_array_equal(perm.cpu().numpy(), ref)
    B = permute_symmetric(Lt, ref)
    rp, ci, va = Ar.export()
    np.testing.assert_array_equal(rp, B.indptr)
    np.testing.assert_array_equal(ci, B.indices)
    assert np.abs(va - B.data).max(initial=0.0) <= assembly_atol(L)


# ------------------------------------------------------------------ SpMV
@pytest.mark.parametrize("Nc,Nm", [(1, 1), (3, 5), (6, 20), (10, 30)])
def test_spmv_matches_oracle(Nc, Nm):
    p = SystemParams(Nc, Nm, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    B = gpu_csr(Ar)
    rng = np.random.default_rng(Nc * 100 + Nm)
    x = rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)
    y = api.spmv(Ar, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = B @ x
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


# ------------------------------------------------------------------ ILU sweeps
@pytest.mark.parametrize("Nc,Nm,d,fill", [(4, 10, 1e-4, 10.0), (3, 5, 0.0, 1e6), (6, 20, 1e-4, 20.0)])
def test_ilu_apply_matches_oracle(Nc, Nm, d, fill):
    p = SystemParams(Nc, Nm, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, d, fill, adjoint=True, fp64_sweeps=True)
    B = gpu_csr(Ar)
    F = ilut(B, d, fill)
    assert M.nnz_l == F.nnz_l and M.nnz_u == F.nnz_u
    rng = np.random.default_rng(7)
    v = rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)
    vt = torch.from_numpy(v).cuda()
    for h in (False, True):
        ref = F.solve_h(v) if h else F.solve(v)
        z = api.ilu_apply(M, vt, conj_transpose=h, fp64=True).cpu().numpy()
        np.testing.assert_allclose(z, ref, rtol=0, atol=1e-10 * np.abs(ref).max())
        # complex64 sweeps: FP32 rounding amplified by the factors' conditioning
        z32 = api.ilu_apply(M, vt, conj_transpose=h, fp64=False).cpu().numpy()
        assert np.abs(z32 - ref).max() <= 1e-3 * np.abs(ref).max()


@pytest.mark.parametrize("Nc,Nm,d,fill", [(4, 10, 1e-4, 10.0), (6, 20, 1e-4, 20.0)])
def test_ilu_condest_matches_oracle(Nc, Nm, d, fill):
    """||(LU)^{-1} e||_inf (Sec. IV) against the oracle's factor solves."""
    p = SystemParams(Nc, Nm, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, d, fill, fp64_sweeps=True)
    F = ilut(gpu_csr(Ar), d, fill)
    ref = np.abs(F.solve(np.ones(Ar.N, dtype=complex))).max()
    assert abs(api.ilu_condest(M, fp64=True) - ref) <= 1e-10 * ref
    assert abs(api.ilu_condest(M) - ref) <= 1e-3 * ref


def test_ilu_condest_flags_the_unstable_fill():
    """The 40,000-row system with the 360,000-row parameters: ILUT(1e-5, 10)
    leaves an unstable factor (estimate overflowing or astronomically large),
    ILUT(1e-5, 100) a usable one -- the reason the solver workload uses p = 100."""
    from paper_1411_4356_gb300 import MID
    A = api.build_liouvillian(MID.params.with_(Nm=20), MID.trace_mode, MID.nth_floor)
    Ar, perm = api.permute(A)
    bad = api.ilu_condest(api.ilu_factor(Ar, MID.droptol, 10.0))
    good = api.ilu_condest(api.ilu_factor(Ar, MID.droptol, MID.fill))
    assert not np.isfinite(bad) or bad > 1e20
    assert np.isfinite(good) and good < 1e12


def test_complete_lu_solves_exactly():
    """d = 0 and no cap: M = A, so M^{-1} (A x) = x."""
    p = SystemParams(3, 5, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, 0.0, 1e6, fp64_sweeps=True)
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)).cuda()
    z = api.ilu_apply(M, api.spmv(Ar, x), fp64=True)
    assert float((z - x).abs().max()) < 1e-9


# ------------------------------------------------------------------ solve
def gpu_solve(w_params, droptol, fill, restart, tol, mode="replace", floor=1e-15):
    A = api.build_liouvillian(w_params, mode, floor)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, droptol, fill)
    rho, info = api.steady_state_solve(Ar, M, perm, restart=restart, tol=tol)
    return rho.cpu().numpy(), info


@pytest.mark.parametrize("mode", ["replace", "add"])
@pytest.mark.parametrize("precond_fp64", [False, True])
def test_tiny_solve_matches_dense_lu(mode, precond_fp64):
    w = TINY
    A = api.build_liouvillian(w.params, mode)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, w.droptol, w.fill, fp64_sweeps=precond_fp64)
    rho, info = api.steady_state_solve(Ar, M, perm, restart=w.restart, tol=w.tol, precond_fp64=precond_fp64)
    rho = rho.cpu().numpy()
    ref = steady_state_dense(oparams(w.params), mode).rho
    assert info.eta <= w.tol
    assert np.abs(rho - ref).max() <= 1e-9
    assert np.abs(np.trace(rho) - 1) < 1e-13


@pytest.mark.parametrize("kw", [dict(g0=0.0), dict(E=0.0), dict(n_th=0.0), dict(Delta=0.7, kappa=0.2)])
def test_solve_special_cases_match_dense(kw):
    p = SystemParams(4, 8, **{**BASE, **kw})
    rho, info = gpu_solve(p, 1e-4, 10.0, 30, 1e-12)
    ref = steady_state_dense(oparams(p)).rho
    assert info.eta <= 1e-12
    assert np.abs(rho - ref).max() <= 1e-9


def test_batched_shape_solve_matches_oracle_iterative():
    """6 x 20 (14,400 rows, the smallest batched system)."""
    p = SystemParams(6, 20, 1.0, -1.3, 0.4, 0.8, 0.2, 1e3, 0.2)
    rho, info = gpu_solve(p, 1e-4, 20.0, 30, 1e-11)
    ref = steady_state_iterative(oparams(p), droptol=1e-4, fill=20.0, restart=50, rtol=1e-14)
    assert ref.converged and info.eta <= 1e-11
    assert np.abs(rho - ref.rho).max() <= 1e-9


def test_observables_kernel():
    p = SystemParams(4, 10, **BASE)
    ref = steady_state_dense(oparams(p)).rho
    na, nb = api.observables(p.Nc, p.Nm, torch.from_numpy(ref).cuda())
    o = observables(oparams(p), ref)
    assert na == pytest.approx(o["n_a"], abs=1e-15)
    assert nb == pytest.approx(o["n_b"], abs=1e-15)


def test_properties_at_larger_size():
    """10 x 20 (40,000 rows): eta by the oracle's own assembly, trace,
    Hermiticity and the exact cavity invariant kappa <n_a> = -2 E Im<a>."""
    p = SystemParams(10, 20, 1.0, -1.0, 0.3, 0.5, 0.3, 1e4, 1.0)
    rho, info = gpu_solve(p, 1e-5, 100.0, 50, 1e-11)
    n = p.n
    x = rho.reshape(-1, order="F")
    L = liouvillian(oparams(p), 1e-15)
    assert oracle_eta(L, x) <= 1e-11
    assert abs(np.trace(rho) - 1) < 1e-12
    assert np.abs(rho - rho.conj().T).max() < 1e-9
    c = np.repeat(np.arange(p.Nc), p.Nm)
    a = np.zeros((n, n))
    for h in range(n):
        if c[h] + 1 < p.Nc:
            a[h, h + p.Nm] = np.sqrt(c[h] + 1)
    na = float(np.real(np.sum(c * np.diag(rho))))
    im_a = float(np.imag(np.trace(a @ rho)))
    assert p.kappa * na == pytest.approx(-2 * p.E * im_a, rel=1e-8, abs=1e-12)


@pytest.mark.parametrize("mode", ["replace", "add"])
def test_single_level_system(mode):
    """The degenerate n = 1 system: L = 0, rho = 1 exactly."""
    p = SystemParams(1, 1, **BASE)
    A = api.build_liouvillian(p, mode)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, 1e-4, 10.0)
    rho, info = api.steady_state_solve(Ar, M, perm, tol=1e-12)
    assert info.status == 0 and abs(complex(rho[0, 0].item()) - 1) < 1e-15


def test_empty_batch():
    rhos, infos = api.steady_state_solve_batched([])
    assert rhos == [] and infos == []
