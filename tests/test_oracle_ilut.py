"""Pins for the oracle's ILUT(d, p) and its triangular sweeps (Sec. II)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle.reorder_factor import ilut


def diag_dominant(rng, n, density):
    """Sparse complex matrix whose columns are strictly diagonally dominant, so
    that Gaussian elimination with partial pivoting picks the diagonal."""
    M = sp.random(n, n, density=density, random_state=rng, format="csr")
    M = M + 1j * sp.random(n, n, density=density, random_state=rng, format="csr")
    M = M.toarray()
    np.fill_diagonal(M, 0)
    colsum = np.abs(M).sum(axis=0)
    M = M + np.diag(colsum + 1.0 + rng.uniform(0, 1, n))
    return sp.csr_matrix(M)


@pytest.mark.parametrize("seed", range(4))
def test_no_dropping_gives_complete_lu(seed):
    """d = 0 and an unbounded fill cap give the complete LU factorisation
    (Sec. II: with d = 0 the iLU returns the complete factorisation)."""
    rng = np.random.default_rng(seed)
    n = 40
    A = diag_dominant(rng, n, 0.08)
    F = ilut(A, 0.0, 1e6)
    P, Lr, Ur = sla.lu(A.toarray())
    np.testing.assert_allclose(P, np.eye(n))  # no pivoting happened in LAPACK either
    np.testing.assert_allclose(F.L().toarray(), Lr, atol=1e-13)
    np.testing.assert_allclose(F.U().toarray(), Ur, atol=1e-13)
    assert F.n_guarded == 0


def test_hand_worked_dropping():
    """A 3x3 case worked by hand.

    A = [[4, 0, 1], [2, 4, 0.01], [0, 1, 4]], d = 0.1, p large.
    Row 1: ||row||_inf = 4, tau = 0.4.  l10 = 2/4 = 0.5 >= tau -> kept;
    w = row1 - 0.5*row0 = [., 4, 0.01 - 0.5] = [., 4, -0.49];  |-0.49| >= 0.4 kept.
    Row 2: tau = 0.4; l21 = 1/4 = 0.25 < tau -> dropped (no elimination);
    u22 = 4.
    """
    A = sp.csr_matrix(np.array([[4, 0, 1], [2, 4, 0.01], [0, 1, 4]], dtype=complex))
    F = ilut(A, 0.1, 100.0)
    np.testing.assert_allclose(F.L().toarray(), [[1, 0, 0], [0.5, 1, 0], [0, 0, 1]])
    np.testing.assert_allclose(F.U().toarray(), [[4, 0, 1], [0, 4, -0.49], [0, 0, 4]])


def test_small_original_entries_are_dropped():
    """Sec. IV: entries below the tolerance are absent from the factors even
    when they are entries of A (the 1e-15 thermal terms)."""
    A = sp.csr_matrix(np.array([[2, 1e-15, 0], [1e-15, 2, 1], [0, 1, 2]], dtype=complex))
    F = ilut(A, 1e-4, 100.0)
    assert 1 not in F.ui[F.up[0]:F.up[1]]
    assert F.nnz_l == 1  # only l21


def test_fill_cap_per_row():
    rng = np.random.default_rng(7)
    A = diag_dominant(rng, 60, 0.15)
    p = 1.0
    F = ilut(A, 0.0, p)
    nnz = np.diff(A.indptr)
    cap = np.maximum(np.floor(p * nnz / 2), 1)
    assert np.all(np.diff(F.lp) <= cap)
    assert np.all(np.diff(F.up) <= cap)
    assert F.nnz_l + F.nnz_u <= p * A.nnz
    # kept entries of each L row are the largest of the unrestricted row
    assert F.fill_factor(A.nnz) <= p


def test_pivot_guard():
    A = sp.csr_matrix(np.array([[1, 1], [1, 1]], dtype=complex))
    F = ilut(A, 0.0, 100.0)
    assert F.n_guarded == 1
    assert abs(F.ux[F.up[1]]) == pytest.approx(1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_sweeps_against_dense_solves(seed):
    rng = np.random.default_rng(seed + 10)
    n = 50
    A = diag_dominant(rng, n, 0.1)
    F = ilut(A, 1e-2, 3.0)
    Ld, Ud = F.L().toarray(), F.U().toarray()
    M = Ld @ Ud
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(F.solve(v), np.linalg.solve(M, v), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(F.solve_h(v), np.linalg.solve(M.conj().T, v), rtol=1e-12, atol=1e-12)


def test_hand_worked_fill_cap_with_ties():
    """The fill cap binding in both parts, worked by hand (Sec. II: keep the
    largest entries; ties go to the smaller column).

    Rows 0-2 are diag(2).  d = 0, p = 0.7.
    Row 3 = [4, 2, 2i, 5, 3, 3i]: nnz 6, cap floor(0.7*6/2) = 2.
      L candidates 2, 1, i (moduli 2, 1, 1): col 0 and, of the tied cols 1
      and 2, col 1.  U: cap - 1 = 1 entry besides the pivot 5; 3 and 3i tie,
      col 4 is kept.
    Row 4 = [1, -3, 0, 2, 6, -4]: nnz 5, cap floor(1.75) = 1.
      Multipliers 0.5, -1.5 (rows 0, 1) and 2/5 = 0.4 (row 3, eliminated
      although the cap drops it later): w4 = 6 - 0.4 * 3 = 4.8, w5 = -4.
      L keeps the largest modulus, col 1 (-1.5, not the largest real part
      0.5); U keeps no entry besides the pivot 4.8.
    Row 5 = e5."""
    A = np.zeros((6, 6), dtype=complex)
    A[0, 0] = A[1, 1] = A[2, 2] = 2
    A[3] = [4, 2, 2j, 5, 3, 3j]
    A[4] = [1, -3, 0, 2, 6, -4]
    A[5, 5] = 1
    F = ilut(sp.csr_matrix(A), 0.0, 0.7)
    Lx = np.zeros((6, 6), dtype=complex)
    Lx[3, 0], Lx[3, 1] = 2, 1
    Lx[4, 1] = -1.5
    Ux = np.diag([2, 2, 2, 5, 4.8, 1]).astype(complex)
    Ux[3, 4] = 3
    np.testing.assert_allclose(F.L().toarray() - np.eye(6), Lx, atol=1e-15)
    np.testing.assert_allclose(F.U().toarray(), Ux, atol=1e-15)
    assert F.n_guarded == 0


# ---- equilibration before the factorisation (the iLUTP of Sec. II as SuperLU runs it)

def test_equilibration_hand_worked():
    """r_i = 1/max_j |a_ij| = (1/4, 2, 1/8); diag(r) A = [[.5, -1, 0], [0, 1, .5],
    [1, 0, .125i]] has column maxima (1, 1, .5), so c = (1, 1, 2)."""
    from oracle.reorder_factor import equilibrate

    A = sp.csr_matrix(np.array([[2, -4, 0], [0, 0.5, 0.25], [8, 0, 1j]], dtype=complex))
    r, c = equilibrate(A)
    np.testing.assert_array_equal(r, [0.25, 2.0, 0.125])
    np.testing.assert_array_equal(c, [1.0, 1.0, 2.0])
    B = (sp.diags(r) @ A @ sp.diags(c)).toarray()
    np.testing.assert_array_equal(B, [[0.5, -1, 0], [0, 1, 1], [1, 0, 0.25j]])


def test_equilibration_maxima_and_empty_lines():
    from oracle.reorder_factor import equilibrate

    rng = np.random.default_rng(9)
    A = sp.random(60, 60, density=0.08, random_state=3, format="csr") * (1 + 1j)
    A = sp.csr_matrix(A + sp.diags(rng.uniform(1e-3, 1e3, 60)))
    A = sp.csr_matrix(sp.diags(10.0 ** rng.uniform(-6, 6, 60)) @ A)
    r, c = equilibrate(A)
    R = abs(sp.diags(r) @ A)
    np.testing.assert_allclose(R.max(axis=1).toarray().ravel(), 1.0, rtol=1e-15)
    B = abs(sp.diags(r) @ A @ sp.diags(c))
    np.testing.assert_allclose(B.max(axis=0).toarray().ravel(), 1.0, rtol=1e-15)
    assert (c >= 1.0).all()
    # a diagonal matrix equilibrates to unit moduli with c = 1
    D = sp.diags(np.array([3.0, -0.5j, 2 + 2j]), format="csr")
    r, c = equilibrate(D)
    np.testing.assert_allclose(r, [1 / 3, 2.0, 1 / np.sqrt(8)], rtol=1e-15)
    np.testing.assert_array_equal(c, 1.0)
    # an empty row and column keep the scale 1
    E = sp.csr_matrix(np.array([[0, 0, 0], [0, 4.0, 0], [0, 0, 0]], dtype=complex))
    r, c = equilibrate(E)
    np.testing.assert_array_equal(r, [1.0, 0.25, 1.0])
    np.testing.assert_array_equal(c, [1.0, 1.0, 1.0])


def test_equilibrated_complete_lu_inverts_the_original_matrix():
    """With no dropping, diag(c) (L U)^{-1} diag(r) v = A^{-1} v: the scalings are
    applied on the right sides (a swapped or missing scaling fails)."""
    from oracle.reorder_factor import equilibrate

    rng = np.random.default_rng(4)
    n = 40
    A = sp.random(n, n, density=0.15, random_state=5, format="csr") * (2 - 1j) + sp.diags(rng.uniform(1, 2, n))
    A = sp.csr_matrix(sp.diags(10.0 ** rng.uniform(-4, 4, n)) @ A @ sp.diags(10.0 ** rng.uniform(-3, 3, n)))
    A.sort_indices()
    r, c = equilibrate(A)
    F = ilut(sp.diags(r) @ A @ sp.diags(c), 0.0, 2.0 * n)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = c * F.solve(r * v)
    ref = np.linalg.solve(A.toarray(), v)
    np.testing.assert_allclose(x, ref, rtol=1e-9, atol=0)


# ---- ILUTP: threshold column pivoting (the "P" of the iLUTP of Sec. II)

def test_ilutp_hand_worked_swap():
    """A = [[1, 4], [2, 3]].  permtol 0.1: 0.1 * 4 < 1, no swap.  permtol 0.5:
    0.5 * 4 > 1, so column 1 takes position 0 (q = [1, 0]), U row 0 = (4, 1);
    row 1 in positions is (3, 2): l = 3/4 and u = 2 - (3/4) 1 = 5/4."""
    from oracle.reorder_factor import ilutp

    A = sp.csr_matrix(np.array([[1, 4], [2, 3]], dtype=complex))
    F = ilutp(A, 0.0, 10.0, 0.1)
    assert F.n_swaps == 0 and list(F.q) == [0, 1]
    F = ilutp(A, 0.0, 10.0, 0.5)
    assert F.n_swaps == 1 and list(F.q) == [1, 0]
    np.testing.assert_allclose(F.U().toarray(), [[4, 1], [0, 1.25]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(F.L().toarray(), [[1, 0], [0.75, 1]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_ilutp_without_pivoting_is_ilut(seed):
    from oracle.reorder_factor import ilutp

    rng = np.random.default_rng(seed)
    A = diag_dominant(rng, 80, 0.06)
    A = sp.csr_matrix(A + sp.random(80, 80, density=0.03, random_state=seed) * 5.0)
    A.sort_indices()
    for d, fill in ((0.0, 1e3), (1e-2, 3.0)):
        F, G = ilut(A, d, fill), ilutp(A, d, fill, 0.0)
        assert G.n_swaps == 0 and list(G.q) == list(range(80))
        for a, b in ((F.lp, G.lp), (F.li, G.li), (F.up, G.up), (F.ui, G.ui)):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(F.lx, G.lx)
        np.testing.assert_array_equal(F.ux, G.ux)


@pytest.mark.parametrize("seed", range(3))
def test_ilutp_complete_factorisation_pivots_by_rows_of_u(seed):
    """d = 0, no cap, permtol = 1: A Q = L U exactly, every U row has its
    largest modulus on the diagonal, and M^{-1} = A^{-1}, also on a matrix
    with zeros on the diagonal."""
    from oracle.reorder_factor import ilutp

    rng = np.random.default_rng(seed)
    n = 30
    A = sp.random(n, n, density=0.2, random_state=seed, format="csr") * (1 + 2j)
    A = A + sp.csr_matrix((rng.uniform(1, 2, n), (np.arange(n), rng.permutation(n))), shape=(n, n))
    A = sp.csr_matrix(A)
    A.setdiag(0)
    A.eliminate_zeros()
    A.sort_indices()
    F = ilutp(A, 0.0, 4.0 * n, 1.0)
    assert F.n_guarded == 0
    Ad = A.toarray()
    LU = F.L().toarray() @ F.U().toarray()
    np.testing.assert_allclose(LU, Ad[:, F.q], rtol=0, atol=1e-12 * np.abs(Ad).max())
    U = F.U().toarray()
    assert (np.abs(np.diag(U))[:, None] >= np.abs(np.triu(U, 1)) * (1 - 1e-15)).all()
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(F.solve(v), np.linalg.solve(Ad, v), rtol=1e-9)
    np.testing.assert_allclose(F.solve_h(v), np.linalg.solve(Ad.conj().T, v), rtol=1e-9)


# ---- the fill cap read as a total, NNZ(L) + NNZ(U) <= p NNZ(A), held as a running budget

def test_total_budget_hand_worked():
    """A = [[2, 0, 0], [1, 2, 0], [3, 1, 2]], d = 0, p = 0.8 (cumulative NNZ 1, 3, 6).
    Row 0 keeps its diagonal (budget floor(0.8) - 0 - 1 < 0).  Row 1: budget
    floor(2.4) - 1 - 1 = 0, so l10 = 0.5 goes.  Row 2: budget floor(4.8) - 2 - 1 = 1;
    its candidates are l20 = 3/2 and l21 = 1/2, and the larger stays."""
    A = sp.csr_matrix(np.array([[2, 0, 0], [1, 2, 0], [3, 1, 2]], dtype=complex))
    F = ilut(A, 0.0, 0.8, cap="total")
    np.testing.assert_array_equal(F.lp, [0, 0, 0, 1])
    np.testing.assert_array_equal(F.li, [0])
    np.testing.assert_allclose(F.lx, [1.5], rtol=0, atol=0)
    np.testing.assert_allclose(np.diag(F.U().toarray()), [2, 2, 2], rtol=0, atol=0)
    assert F.nnz_l + F.nnz_u <= 0.8 * A.nnz + 3


@pytest.mark.parametrize("seed", range(3))
def test_total_budget_that_never_binds_is_threshold_ilu(seed):
    """With a budget above the natural fill, cap="total" keeps every entry that
    survives the drop rule: the same factors as a per-row cap that never binds."""
    rng = np.random.default_rng(seed)
    A = diag_dominant(rng, 80, 0.06)
    A = sp.csr_matrix(A + sp.random(80, 80, density=0.03, random_state=seed) * 5.0)
    A.sort_indices()
    for d in (0.0, 1e-2):
        F, G = ilut(A, d, 200.0), ilut(A, d, 200.0, cap="total")
        assert F.nnz_l + F.nnz_u < 200.0 * A.nnz / 4
        for a, b in ((F.lp, G.lp), (F.li, G.li), (F.up, G.up), (F.ui, G.ui)):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(F.lx, G.lx)
        np.testing.assert_array_equal(F.ux, G.ux)


def test_total_budget_bounds_the_fill():
    rng = np.random.default_rng(7)
    A = diag_dominant(rng, 120, 0.05)
    for p in (1.0, 1.5, 3.0):
        F = ilut(A, 0.0, p, cap="total")
        assert F.nnz_l + F.nnz_u <= np.floor(p * A.nnz) + 0  # diagonal included in the count
