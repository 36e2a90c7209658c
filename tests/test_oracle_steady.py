"""Pins for the oracle's GMRES, steady state and adjoint against closed forms,
exact invariants and independent solvers."""
import numpy as np
import pytest
import scipy.sparse as sp
from math import factorial

from oracle.gmres import gmres_right
from oracle.liouvillian import Params, mode_operators
from oracle.steady import (THETAS, adjoint_gradient_dense, adjoint_gradient_iterative, expect,
                           number_operators, observable_vec, observables, steady_observable,
                           steady_state_dense, steady_state_iterative)

TINY = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


# ---------------------------------------------------------------- GMRES
@pytest.mark.parametrize("restart", [3, 10, 40])
def test_gmres_matches_direct_solve(restart):
    rng = np.random.default_rng(restart)
    n = 40
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3 + 1j * rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    r = gmres_right(lambda v: A @ v, lambda v: v, b, restart=restart, rtol=1e-13)
    assert r.converged
    np.testing.assert_allclose(r.x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-11)


def test_gmres_exact_preconditioner_one_step():
    rng = np.random.default_rng(5)
    n = 30
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 5 * np.eye(n)
    Ainv = np.linalg.inv(A)
    b = rng.standard_normal(n) + 0j
    r = gmres_right(lambda v: A @ v, lambda v: Ainv @ v, b, restart=10, rtol=1e-12)
    assert r.converged and r.iterations == 1


# ---------------------------------------------------------------- closed forms
def thermal(Nm, nth):
    r = nth / (1 + nth)
    k = np.arange(Nm)
    return r ** k * (1 - r) / (1 - r ** Nm)


def coherent(Nc, alpha):
    c = np.arange(Nc)
    amp = np.array([alpha ** k / np.sqrt(float(factorial(k))) for k in c]) * np.exp(-abs(alpha) ** 2 / 2)
    return amp


def test_g0_zero_product_of_coherent_and_thermal():
    """g0 = 0 decouples the modes: the cavity is the coherent state
    alpha = -iE / (kappa/2 - i Delta) and the mechanics the thermal state of
    occupation n_th (exact under truncation by detailed balance)."""
    # N_c = 14 puts the truncated coherent tail (|alpha|^13 / sqrt(13!)) below 1e-14
    p = Params(14, 4, omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.0, E=0.2, Q_m=1e3, n_th=0.5)
    rho = steady_state_dense(p).rho
    alpha = -1j * p.E / (p.kappa / 2 - 1j * p.Delta)
    psi = coherent(p.Nc, alpha)
    rc = np.outer(psi, psi.conj())
    rm = np.diag(thermal(p.Nm, p.n_th))
    np.testing.assert_allclose(rho, np.kron(rc, rm), atol=1e-13)


def test_e_zero_vacuum_times_thermal():
    """E = 0: the cavity relaxes to vacuum and the mechanics to the thermal state, for any g0."""
    p = Params(4, 8, omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.7, E=0.0, Q_m=1e3, n_th=0.8)
    rho = steady_state_dense(p).rho
    rc = np.zeros((p.Nc, p.Nc))
    rc[0, 0] = 1.0
    np.testing.assert_allclose(rho, np.kron(rc, np.diag(thermal(p.Nm, p.n_th))), atol=1e-13)


def test_exact_invariants_under_truncation():
    """From Tr(N L rho) = 0 with the truncated [N, a] = -a:
    kappa <a^dag a> = -2 E Im<a>;
    -2 g0 Im<a^dag a b> - Gamma_m (1 + n_th) <b^dag b> + Gamma_m n_th <b b^dag>_trunc = 0;
    plus Tr rho = 1, rho = rho^H, rho >= 0."""
    p = Params(4, 10, **TINY)
    rho = steady_state_dense(p).rho
    a, b = mode_operators(p.Nc, p.Nm)
    na, nb = number_operators(p)
    Gm = p.omega_m / p.Q_m
    assert p.kappa * expect(na, rho).real == pytest.approx(-2 * p.E * expect(a, rho).imag, abs=1e-15)
    bbd = (b @ b.conj().T).tocsr()
    bal = (-2 * p.g0 * expect(na @ b, rho).imag - Gm * (1 + p.n_th) * expect(nb, rho).real
           + Gm * p.n_th * expect(bbd, rho).real)
    assert abs(bal) < 1e-14
    assert np.trace(rho) == pytest.approx(1.0, abs=1e-14)
    np.testing.assert_allclose(rho, rho.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh((rho + rho.conj().T) / 2).min() > -1e-13


def test_trace_modes_agree():
    p = Params(4, 10, **TINY)
    np.testing.assert_allclose(steady_state_dense(p, "add").rho, steady_state_dense(p, "replace").rho,
                               atol=1e-13)


def test_zero_temperature_floor_leaves_solution_unchanged():
    """Sec. IV: n_th = 1e-15 gives a density matrix numerically identical to n_th = 0."""
    p = Params(4, 10, **{**TINY, "n_th": 0.0})
    r0 = steady_state_dense(p, nth_floor=0.0).rho
    r1 = steady_state_dense(p, nth_floor=1e-15).rho
    np.testing.assert_allclose(r0, r1, atol=1e-12)


@pytest.mark.parametrize("mode", ["replace", "add"])
def test_iterative_pipeline_matches_dense(mode):
    """Sec. IV: converged to machine precision, the RCM-ILUT-GMRES answer is
    numerically identical to direct LU."""
    p = Params(4, 10, **TINY)
    d = steady_state_dense(p, mode)
    it = steady_state_iterative(p, mode, droptol=1e-4, fill=10.0, restart=30, rtol=1e-14)
    assert it.converged
    np.testing.assert_allclose(it.rho, d.rho, atol=1e-12)
    assert it.eta < 1e-13


# ---------------------------------------------------------------- adjoint
def fd_grad(p, which, theta, h, mode):
    up = Params(**{**p.__dict__, theta: getattr(p, theta) + h})
    dn = Params(**{**p.__dict__, theta: getattr(p, theta) - h})
    return (steady_observable(up, which, mode) - steady_observable(dn, which, mode)) / (2 * h)


@pytest.mark.parametrize("mode", ["replace", "add"])
@pytest.mark.parametrize("which", ["n_a", "n_b"])
def test_adjoint_matches_central_differences(mode, which):
    """Central differences with Richardson extrapolation (h = 1e-4, 5e-5):
    truncation error O(h^4) ~ 1e-10 relative, solve round-off ~ 1e-8."""
    p = Params(3, 8, **TINY)
    g = adjoint_gradient_dense(p, observable_vec(p, which), mode)
    for t in THETAS:
        d1 = fd_grad(p, which, t, 1e-4, mode)
        d2 = fd_grad(p, which, t, 5e-5, mode)
        fd = (4 * d2 - d1) / 3
        assert g[t] == pytest.approx(fd, rel=1e-7, abs=1e-11), (t, g[t], fd)


def test_adjoint_iterative_matches_dense():
    p = Params(4, 10, **TINY)
    G = observable_vec(p, "n_b")
    gd = adjoint_gradient_dense(p, G)
    gi = adjoint_gradient_iterative(p, G, droptol=1e-4, fill=10.0, restart=30)
    for t in THETAS:
        assert gi[t] == pytest.approx(gd[t], rel=1e-9, abs=1e-13)


def test_observables_definition():
    p = Params(3, 4, **TINY)
    rho = steady_state_dense(p).rho
    o = observables(p, rho)
    c = np.repeat(np.arange(p.Nc), p.Nm)
    m = np.tile(np.arange(p.Nm), p.Nc)
    assert o["n_a"] == pytest.approx(float(np.real(np.sum(c * np.diag(rho)))), abs=1e-15)
    assert o["n_b"] == pytest.approx(float(np.real(np.sum(m * np.diag(rho)))), abs=1e-15)


@pytest.mark.parametrize("mode", ["replace", "add"])
def test_single_level_system_has_rho_one(mode):
    """n = 1 (N_c = N_m = 1): L = 0, so the trace condition alone fixes rho = 1."""
    from oracle.liouvillian import Params
    p = Params(1, 1, 1.0, -1.0, 0.5, 0.3, 0.2, 1e3, 0.5)
    r = steady_state_dense(p, mode)
    assert r.rho.shape == (1, 1) and abs(r.rho[0, 0] - 1) < 1e-15


def test_eta_hand_value():
    """eta = ||L x||_inf / (||L||_inf ||x||_inf), worked by hand on a 3 x 3 L.

    L = [[1, -2, 0], [0, 3, i], [2, 0, -1]], x = (1, i, -1):
    L x = (1 - 2i, 2i, 3) -> ||L x||_inf = 3 (a 2-norm would give sqrt(18));
    row sums of |L| are 3, 4, 3 -> ||L||_inf = 4; ||x||_inf = 1; eta = 0.75."""
    import scipy.sparse as sp

    from oracle.steady import eta

    L = sp.csr_matrix(np.array([[1, -2, 0], [0, 3, 1j], [2, 0, -1]], dtype=complex))
    x = np.array([1, 1j, -1], dtype=complex)
    assert eta(L, x) == pytest.approx(0.75, rel=1e-15)
    assert eta(L, 4 * x) == pytest.approx(0.75, rel=1e-15)  # scale invariant


def test_dense_eta_uses_the_unmodified_liouvillian():
    """The reported residual is that of L, not of L~: with the trace row the
    converged x would leave L~ x - 0 = w e_0, an eta near |w| / ||L~||."""
    from oracle.liouvillian import augmented

    p = Params(3, 4, 1.0, -1.0, 0.5, 0.3, 0.2, 1e3, 0.5)
    r = steady_state_dense(p)
    Lt, b, w, L = augmented(p)
    assert r.eta < 1e-14
    lt_inf = np.abs(Lt).sum(axis=1).max()
    assert np.abs(Lt @ r.x).max() / (lt_inf * np.abs(r.x).max()) > 1e-4


def test_phonon_distribution_thermal_closed_form():
    """g0 = 0: the mechanics is the truncated thermal state, P(m) = r^m (1 - r) /
    (1 - r^N_m), r = n_th / (1 + n_th) (exact under truncation by detailed
    balance); its Fano factor follows from the same closed form."""
    from oracle.steady import fano_factor, phonon_distribution

    p = Params(3, 12, 1.0, -1.0, 0.5, 0.0, 0.2, 1e3, 1.5)
    rho = steady_state_dense(p).rho
    r = p.n_th / (1 + p.n_th)
    m = np.arange(p.Nm)
    P = r ** m * (1 - r) / (1 - r ** p.Nm)
    np.testing.assert_allclose(phonon_distribution(p, rho), P, atol=1e-12)
    mean = (m * P).sum()
    F = ((m * m * P).sum() - mean ** 2) / mean
    assert fano_factor(phonon_distribution(p, rho)) == pytest.approx(F, rel=1e-10)
    # the distribution sums to Tr rho = 1, and its mean is <b^dag b>
    assert phonon_distribution(p, rho).sum() == pytest.approx(1.0, abs=1e-13)
    assert mean == pytest.approx(observables(p, rho)["n_b"], rel=1e-11)


def test_fano_factor_of_a_fock_and_a_poisson_distribution():
    from oracle.steady import fano_factor

    P = np.zeros(8)
    P[3] = 1.0
    assert fano_factor(P) == pytest.approx(0.0, abs=1e-15)
    lam = 2.0
    k = np.arange(60)
    from math import lgamma

    Q = np.exp(k * np.log(lam) - lam - np.array([lgamma(x + 1) for x in k]))
    assert fano_factor(Q) == pytest.approx(1.0, rel=1e-12)
