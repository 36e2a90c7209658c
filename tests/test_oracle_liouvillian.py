"""Pins for the oracle's Liouvillian (Eq. 1, 3, 4, 5) against facts fixed by
the paper and by the mathematics, not by the oracle itself."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.liouvillian import (Params, augmented, bandwidth_profile, diagonal_positions,
                                liouvillian, liouvillian_row, superoperator_column,
                                trace_weight)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TINY = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


def test_nnz_matches_fig1():
    """Fig. 1: NNZ(L~) = 8957 at N_c = 4, N_m = 8 with a thermal bath (Eq. 5 adds w T)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_fig1.json")))
    p = Params(g["Nc"], g["Nm"], **TINY)
    Lt, _, _, _ = augmented(p, g["trace_mode"])
    assert Lt.nnz == g["nnz"]
    # the replace reading drops the two row-0 entries of L that sit on diagonal columns
    Lr, _, _, _ = augmented(p, "replace")
    assert Lr.nnz == g["nnz"] - 2


def test_columns_equal_superoperator_action():
    """Brute force: column k of the Kronecker-form matrix equals vec(L[E_ij])
    with L applied by dense matrix products (Eq. 3), k = i + j n (Eq. 4)."""
    p = Params(3, 4, **TINY)
    L = liouvillian(p).toarray()
    for k in range(L.shape[0]):
        np.testing.assert_allclose(L[:, k], superoperator_column(p, k), rtol=0, atol=1e-14)


def test_row_extractor_matches_assembly():
    p = Params(4, 6, **TINY)
    L = liouvillian(p)
    rng = np.random.default_rng(0)
    for k in rng.choice(L.shape[0], 30, replace=False):
        cols, vals = liouvillian_row(p, int(k))
        row = L.getrow(int(k))
        np.testing.assert_array_equal(cols, row.indices)
        np.testing.assert_allclose(vals, row.data, rtol=0, atol=1e-14)


def test_trace_and_hermiticity_preserving():
    """Lindblad form: Tr(L rho) = 0 for every rho, i.e. the rows at the
    diagonal positions sum to zero, and L maps Hermitian to Hermitian."""
    p = Params(4, 5, **TINY)
    n = p.Nc * p.Nm
    L = liouvillian(p)
    s = np.asarray(L[diagonal_positions(n)].sum(axis=0)).ravel()
    assert np.abs(s).max() < 1e-13
    rng = np.random.default_rng(1)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    X = X + X.conj().T
    Y = (L @ X.reshape(-1, order="F")).reshape((n, n), order="F")
    np.testing.assert_allclose(Y, Y.conj().T, atol=1e-12)


def test_trace_weight_closed_form():
    """mean diag(L) = -(1/n) sum_O gamma_O Tr(O^dag O)
    = -[kappa (N_c - 1) + Gamma_m (1 + 2 n_th)(N_m - 1)] / 2 (truncated traces)."""
    for Nc, Nm in [(4, 10), (3, 7), (6, 20)]:
        p = Params(Nc, Nm, **TINY)
        Gm = p.omega_m / p.Q_m
        expected = -(p.kappa * (Nc - 1) + Gm * (1 + 2 * p.n_th) * (Nm - 1)) / 2
        assert trace_weight(liouvillian(p)) == pytest.approx(expected, rel=1e-13)


def test_stencil_size_and_value_independent_structure():
    """At most 9 Hamiltonian + 3 jump entries per row; the structure does not
    depend on the (nonzero) values of Delta, E, g0, kappa."""
    p = Params(4, 10, **TINY)
    L = liouvillian(p)
    assert np.diff(L.indptr).max() <= 12
    q = Params(4, 10, omega_m=1.0, Delta=-2.3, kappa=0.17, g0=1.1, E=0.9, Q_m=1e4, n_th=3.0)
    L2 = liouvillian(q)
    np.testing.assert_array_equal(L.indptr, L2.indptr)
    np.testing.assert_array_equal(L.indices, L2.indices)


def test_trace_row_bandwidth():
    """Sec. III: T makes the upper bandwidth n^2 - 1 (it has an entry in the final
    column, Sec. II), so B(L~) > (N_c N_m)^2."""
    p = Params(4, 8, **TINY)
    n = p.Nc * p.Nm
    for mode in ("add", "replace"):
        Lt, b, w, _ = augmented(p, mode)
        bp = bandwidth_profile(Lt)
        assert bp["ub"] == n * n - 1
        assert bp["B"] > n * n
        assert b[0] == w and np.all(b[1:] == 0)


def test_replace_row_is_trace_functional():
    p = Params(3, 5, **TINY)
    n = p.Nc * p.Nm
    Lt, b, w, L = augmented(p, "replace")
    row0 = Lt.getrow(0)
    np.testing.assert_array_equal(row0.indices, diagonal_positions(n))
    np.testing.assert_array_equal(row0.data, np.full(n, w))
    # rows >= 1 are those of L
    D = (Lt - L)[1:]
    assert abs(D).max() == 0


def test_nth_floor_only_at_zero_temperature():
    """Sec. IV: n_th = 1e-15 keeps the thermal entries in the structure."""
    p0 = Params(4, 10, **{**TINY, "n_th": 0.0})
    assert liouvillian(p0, 0.0).nnz < liouvillian(p0, 1e-15).nnz
    assert liouvillian(p0, 1e-15).nnz == liouvillian(Params(4, 10, **TINY)).nnz
    p1 = Params(4, 10, **TINY)
    assert (liouvillian(p1, 1e-15) != liouvillian(p1, 0.0)).nnz == 0


def test_bandwidth_profile_definition():
    """Sec. II definitions on a hand-made matrix."""
    A = sp.csr_matrix(np.array([[1, 0, 2, 0],
                                [0, 1, 0, 0],
                                [3, 0, 1, 4],
                                [0, 5, 0, 1]], dtype=complex))
    bp = bandwidth_profile(A)
    assert (bp["ub"], bp["lb"]) == (2, 2)
    assert bp["B"] == 5
    assert bp["up"] == 2 + 0 + 1 + 0
    assert bp["lp"] == 2 + 2 + 0 + 0


# ---- Hamiltonian variants of Sec. VI: g2 (b + b^dag)^2 a^dag a and lam (b + b^dag)^4

def _mech_block(p, c):
    """The mechanical block <c, m| H |c, m'> of the oracle's H at cavity level c."""
    from oracle.liouvillian import hamiltonian

    H = hamiltonian(p).toarray()
    s = slice(c * p.Nm, (c + 1) * p.Nm)
    return H[s, s]


def test_powers_of_position_match_the_ladder_closed_forms():
    """Away from the cutoff, <m|X^2|m> = 2m + 1, <m+2|X^2|m> = sqrt((m+1)(m+2)),
    <m|X^4|m> = 6m^2 + 6m + 3, <m+2|X^4|m> = (4m + 6) sqrt((m+1)(m+2)) and
    <m+4|X^4|m> = sqrt((m+1)(m+2)(m+3)(m+4)) (X = b + b^dag, from b|m> =
    sqrt(m)|m-1>): the g2 term at c = 1 and the lam term at c = 0."""
    Nm = 24
    base = dict(omega_m=0.0, Delta=0.0, kappa=0.1, g0=0.0, E=0.0, Q_m=1e3, n_th=0.0)
    X2 = _mech_block(Params(2, Nm, **base, g2=1.0), 1)
    X4 = _mech_block(Params(1, Nm, **base, lam=1.0), 0)
    for m in range(Nm - 5):
        assert X2[m, m] == pytest.approx(2 * m + 1, abs=1e-12)
        assert X2[m + 2, m] == pytest.approx(np.sqrt((m + 1) * (m + 2)), abs=1e-12)
        assert X2[m + 1, m] == 0 and X2[m + 3, m] == 0
        assert X4[m, m] == pytest.approx(6 * m * m + 6 * m + 3, abs=1e-10)
        assert X4[m + 2, m] == pytest.approx((4 * m + 6) * np.sqrt((m + 1) * (m + 2)), abs=1e-10)
        assert X4[m + 4, m] == pytest.approx(np.sqrt((m + 1) * (m + 2) * (m + 3) * (m + 4)), abs=1e-10)
        assert X4[m + 1, m] == 0 and X4[m + 3, m] == 0
    # at the cutoff the truncated square lacks the b b^dag part: <N_m-1|X^2|N_m-1> = N_m - 1
    assert X2[Nm - 1, Nm - 1] == pytest.approx(Nm - 1, abs=1e-12)


def test_quadratic_coupling_shifts_the_mechanical_frequency():
    """omega b^dag b + g2 c X^2 is a harmonic oscillator of frequency
    Omega = sqrt(omega (omega + 4 g2 c)) with levels Omega (k + 1/2) - omega/2
    (x = X / sqrt 2, p^2 + x^2 = 2 b^dag b + 1); the lowest levels of a wide
    truncation reach them.  The cavity term -Delta c is a constant shift."""
    Nm, g2, Delta = 160, 0.15, -0.4
    p = Params(3, Nm, omega_m=1.0, Delta=Delta, kappa=0.1, g0=0.0, E=0.0, Q_m=1e3, n_th=0.0, g2=g2)
    for c in (1, 2):
        ev = np.linalg.eigvalsh(_mech_block(p, c))[:6]
        Om = np.sqrt(1.0 * (1.0 + 4 * g2 * c))
        ref = Om * (np.arange(6) + 0.5) - 0.5 - Delta * c
        np.testing.assert_allclose(ev, ref, rtol=0, atol=1e-9)


def test_variants_enter_the_superoperator_columns():
    """The Kronecker-form L with both variants on against dense products on E_ij."""
    p = Params(3, 6, **TINY, g2=0.07, lam=0.01)
    L = liouvillian(p).toarray()
    for k in range(0, L.shape[0], 7):
        np.testing.assert_allclose(L[:, k], superoperator_column(p, k), rtol=0, atol=1e-13)
