"""The library's host factorisation (om_ilu_factor_host: the ILUT, total-budget
ILUT, ILUTP and equilibration code of om_ilu_factor, run on host arrays with
no device) against the oracle on the RCM-ordered Liouvillian.  No GPU needed.

Structure (row pointers, columns, the pivot permutation) bit-exact; values
within 1e-12 of the largest entry of each factor (the two eliminate in the
same order, with differently grouped complex products); equilibration
scalings within 4 ulp (r |a| on one side, |r a| on the other)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.liouvillian import Params, augmented
from oracle.reorder_factor import equilibrate, ilut, ilutp, permute_symmetric, rcm_permutation
from paper_1411_4356_gb300 import api

BASE = (1.0, -1.0, 0.5, 0.3, 0.2, 1e3, 0.5)
FIG4 = (1.0, -1.0, 0.2, 0.5, 0.1, 1e4, 3.0)


def rcm_matrix(Nc, Nm, prm, floor=1e-15):
    Lt, *_ = augmented(Params(Nc, Nm, *prm), "replace", floor)
    A = sp.csr_matrix(permute_symmetric(Lt, rcm_permutation(Lt)))
    A.sort_indices()
    return A


def oracle_parts(F):
    """Strict U and the diagonal from the oracle's U rows (diagonal first)."""
    n = F.n
    diag = np.array([F.ux[F.up[i]] for i in range(n)])
    counts = np.diff(F.up) - 1
    up = np.concatenate([[0], np.cumsum(counts)])
    keep = np.ones(len(F.ui), dtype=bool)
    keep[F.up[:-1]] = False
    return up, F.ui[keep], F.ux[keep], diag


def compare(H, F):
    np.testing.assert_array_equal(H["lp"], F.lp)
    np.testing.assert_array_equal(H["li"], F.li)
    up, ui, ux, diag = oracle_parts(F)
    np.testing.assert_array_equal(H["up"], up)
    np.testing.assert_array_equal(H["ui"], ui)
    for a, b in ((H["lx"], F.lx), (H["ux"], ux), (H["diag"], diag)):
        if len(b):
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert H["n_guarded"] == F.n_guarded


@pytest.mark.parametrize("Nc,Nm,prm,d,fill", [(4, 10, BASE, 1e-4, 10.0), (6, 20, BASE, 1e-5, 30.0),
                                              (4, 30, FIG4, 1e-4, 100.0)])
def test_row_cap_ilut(Nc, Nm, prm, d, fill):
    A = rcm_matrix(Nc, Nm, prm)
    H = api.ilu_factor_host(A.indptr, A.indices, A.data, d, fill)
    compare(H, ilut(A, d, fill))
    np.testing.assert_array_equal(H["q"], np.arange(A.shape[0]))


@pytest.mark.parametrize("Nc,Nm,prm,d,fill", [(4, 10, BASE, 1e-4, 3.0), (6, 20, BASE, 1e-5, 8.0),
                                              (4, 30, FIG4, 1e-4, 100.0)])
def test_total_budget_ilut(Nc, Nm, prm, d, fill):
    A = rcm_matrix(Nc, Nm, prm, floor=0.0)
    H = api.ilu_factor_host(A.indptr, A.indices, A.data, d, fill, cap="total")
    compare(H, ilut(A, d, fill, cap="total"))


@pytest.mark.parametrize("Nc,Nm,prm,d,fill,permtol", [(3, 5, BASE, 1e-4, 10.0, 0.1), (4, 10, BASE, 1e-4, 10.0, 1.0),
                                                      (4, 20, FIG4, 1e-4, 100.0, 0.1)])
@pytest.mark.parametrize("eq", [False, True])
def test_ilutp_and_equilibration(Nc, Nm, prm, d, fill, permtol, eq):
    A = rcm_matrix(Nc, Nm, prm, floor=0.0)
    H = api.ilu_factor_host(A.indptr, A.indices, A.data, d, fill, permtol=permtol, equilibrate=eq)
    B = A
    if eq:
        r, c = equilibrate(A)
        np.testing.assert_allclose(H["r"], r, rtol=1e-15, atol=0)
        np.testing.assert_allclose(H["c"], c, rtol=1e-15, atol=0)
        B = sp.csr_matrix(sp.diags(r) @ A @ sp.diags(c))
    F = ilutp(B, d, fill, permtol)
    np.testing.assert_array_equal(H["q"], F.q)
    assert H["n_swaps"] == F.n_swaps
    compare(H, F)


def test_bad_options_are_rejected():
    from paper_1411_4356_gb300._lib import OMError

    A = rcm_matrix(2, 3, BASE)
    with pytest.raises(OMError):
        api.ilu_factor_host(A.indptr, A.indices, A.data, 1e-4, 10.0, permtol=0.1, cap="total")
    with pytest.raises(OMError):
        api.ilu_factor_host(A.indptr, A.indices, A.data, 1e-4, 10.0, permtol=1.5)


@pytest.mark.parametrize("Nc,Nm,prm,floor", [(1, 1, BASE, 1e-15), (2, 3, BASE, 1e-15), (4, 8, BASE, 1e-15),
                                             (10, 20, BASE, 1e-15), (4, 60, FIG4, 0.0), (12, 30, BASE, 1e-15)])
@pytest.mark.parametrize("mode", ["replace", "add"])
def test_host_rcm_order(Nc, Nm, prm, floor, mode):
    """The library's serial RCM walk against the oracle's, bit-exact, up to 129,600 rows."""
    Lt, *_ = augmented(Params(Nc, Nm, *prm), mode, floor)
    Lt = sp.csr_matrix(Lt)
    Lt.sort_indices()
    np.testing.assert_array_equal(api.rcm_order_host(Lt.indptr, Lt.indices), rcm_permutation(Lt))
