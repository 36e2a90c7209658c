"""Pins for the oracle's no-jump operator S (rho -> K rho + rho K^dag) and its
inverse, the second preconditioner of the GPU path.

S is tied to the Liouvillian of Eq. 3 (itself pinned by Fig. 1's NNZ and by
brute-force superoperator columns) through L = S + sum gamma conj(O) (x) O,
to dense matrix products on basis matrices, to a closed form when K is
diagonal, and its inverse to a second, independent route (dense LU of the
Kronecker-sum matrix against the Bartels-Stewart solve).
"""
import numpy as np
import pytest

from oracle.liouvillian import Params, liouvillian
from oracle.nojump import (effective_hamiltonian, jump_operator, nojump_operator, nojump_solve,
                           nojump_solve_dense, steady_state_nojump)
from oracle.steady import steady_state_dense

CASES = [
    Params(3, 4, 1.0, -1.0, 0.5, 0.3, 0.2, 1e3, 0.5),
    Params(2, 5, 1.0, 0.7, 0.3, 0.9, 0.4, 1e2, 2.0),
    Params(4, 3, 1.0, -2.0, 0.4, 0.8, 0.2, 1e3, 0.0),  # n_th = 0, floored
    Params(3, 6, 1.0, -1.0, 0.5, 0.3, 0.2, 1e3, 0.5, g2=0.05, lam=0.01),  # Sec. VI variants
]


@pytest.mark.parametrize("p", CASES)
def test_liouvillian_is_nojump_plus_jumps(p):
    """Eq. 3: L = S + sum_O gamma_O conj(O) (x) O, entry by entry."""
    L = liouvillian(p, 1e-15)
    R = (nojump_operator(p) + jump_operator(p) - L).toarray()
    assert np.abs(R).max() <= 1e-13 * max(1.0, abs(L).max())


@pytest.mark.parametrize("p", CASES[:2])
def test_columns_are_dense_products(p):
    """Column k = i + j n of S is vec(K E_ij + E_ij K^dag) by dense products (Eq. 4)."""
    n = p.Nc * p.Nm
    K = effective_hamiltonian(p)
    S = nojump_operator(p).toarray()
    for k in [0, 1, n, n + 1, n * n - 1, (n * n) // 3]:
        i, j = k % n, k // n
        E = np.zeros((n, n), dtype=complex)
        E[i, j] = 1.0
        col = (K @ E + E @ K.conj().T).reshape(-1, order="F")
        np.testing.assert_allclose(S[:, k], col, atol=1e-15)


def test_closed_form_when_K_is_diagonal():
    """g0 = E = 0: H is diagonal, so X_ij = Y_ij / (K_ii + conj(K_jj)) with
    K_ii = -i(-Delta c + omega_m m) - (kappa c + Gm(1+nth) m + Gm nth (m+1)[m < Nm-1]) / 2."""
    p = Params(3, 5, 1.0, -0.7, 0.4, 0.0, 0.0, 50.0, 1.5)
    n = p.Nc * p.Nm
    Gm = p.omega_m / p.Q_m
    c = np.repeat(np.arange(p.Nc), p.Nm)
    m = np.tile(np.arange(p.Nm), p.Nc)
    bbd = np.where(m < p.Nm - 1, m + 1, 0)  # b b^dag in the truncated space
    k = -1j * (-p.Delta * c + p.omega_m * m) - 0.5 * (p.kappa * c + Gm * (1 + p.n_th) * m + Gm * p.n_th * bbd)
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    X = Y / (k[:, None] + k.conj()[None, :])
    got = nojump_solve(p, Y.reshape(-1, order="F")).reshape((n, n), order="F")
    np.testing.assert_allclose(got, X, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(np.diag(effective_hamiltonian(p)), k, atol=1e-15)


@pytest.mark.parametrize("p", CASES)
@pytest.mark.parametrize("adjoint", [False, True])
def test_sylvester_solve_matches_dense_lu(p, adjoint):
    n = p.Nc * p.Nm
    rng = np.random.default_rng(11)
    y = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    a = nojump_solve(p, y, adjoint=adjoint)
    b = nojump_solve_dense(p, y, adjoint=adjoint)
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12 * np.abs(b).max())


def test_adjoint_is_the_frobenius_adjoint():
    """<S^{-1} Y, X> = <Y, S^{-H} X> in the Frobenius inner product."""
    p = CASES[0]
    n = p.Nc * p.Nm
    rng = np.random.default_rng(5)
    y = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    x = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    lhs = np.vdot(nojump_solve(p, y), x)
    rhs = np.vdot(y, nojump_solve(p, x, adjoint=True))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_hermitian_maps_to_hermitian():
    """S(X)^dag = S(X^dag), so S^{-1} keeps Hermitian matrices Hermitian."""
    p = CASES[1]
    n = p.Nc * p.Nm
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Y = Y + Y.conj().T
    X = nojump_solve(p, Y.reshape(-1, order="F")).reshape((n, n), order="F")
    np.testing.assert_allclose(X, X.conj().T, atol=1e-12 * np.abs(X).max())


@pytest.mark.parametrize("mode", ["replace", "add"])
def test_nojump_preconditioned_gmres_gives_the_steady_state(mode):
    """Right preconditioning by S^{-1} changes the iteration, not the answer of Eq. 5."""
    p = Params(4, 10, 1.0, -1.0, 0.5, 0.3, 0.2, 1e3, 0.5)
    x, its, ok, _ = steady_state_nojump(p, mode, restart=30, rtol=1e-14)
    ref = steady_state_dense(p, mode)
    assert ok
    assert np.abs(x - ref.x).max() <= 1e-11


@pytest.mark.parametrize("m,n", [(37, 37), (300, 300), (300, 170), (90, 410)])
def test_block_recursion_matches_lapack(m, n):
    """The block recursion of the triangular Sylvester solve against LAPACK's
    unblocked ztrsyl on the whole system, and by its residual."""
    import scipy.linalg as sla

    from oracle.nojump import triangular_sylvester

    rng = np.random.default_rng(m * 1000 + n)
    T1 = np.triu(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) + np.diag(-2.0 + 1j * np.arange(m))
    T2 = np.triu(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) + np.diag(-1.5 - 0.5j * np.arange(n))
    Y = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    X = triangular_sylvester(T1, T2, Y, base=32)
    R, scale, info = sla.lapack.ztrsyl(T1, T2, Y, trana="N", tranb="C", isgn=1)
    np.testing.assert_allclose(X, R / scale, rtol=1e-9, atol=1e-12 * np.abs(R).max())
    assert np.abs(T1 @ X + X @ T2.conj().T - Y).max() <= 1e-10 * np.abs(Y).max()
