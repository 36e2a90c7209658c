"""Oracle: the steady state rho_ss of Eq. 2, its residual, observables and the
adjoint gradient.

Test infrastructure only (see ``oracle/__init__.py``).

The result the method computes has a plain definition: the solution x of the
trace-augmented system L~ x = (w, 0, ...)^T of Eq. 5, read as the column-
stacked density matrix (Eq. 4) and normalised to unit trace.  Sec. IV runs
the iterative solver to machine precision, where its answer is numerically
identical to the direct-LU one.  So:

* ``steady_state_dense`` -- dense LU (LAPACK) of L~ on small sizes: the
  definition written out;
* ``steady_state_iterative`` -- the paper's own pipeline on larger sizes:
  RCM (Sec. III) -> ILUT (Sec. II) -> restarted GMRES (Sec. IV), converged
  far below the tolerance of the GPU path.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .gmres import gmres_right
from .liouvillian import Params, augmented, diagonal_positions, mode_operators
from .reorder_factor import equilibrate, ilut, permute_symmetric, rcm_permutation


def rho_from_vec(x: np.ndarray, n: int) -> np.ndarray:
    """Undo the column stacking of Eq. 4: rho[i, j] = x[i + j n]."""
    return np.asarray(x).reshape((n, n), order="F")


def trace_normalise(x: np.ndarray, n: int) -> np.ndarray:
    return x / x[diagonal_positions(n)].sum()


def eta(L: sp.csr_matrix, x: np.ndarray) -> float:
    """Normwise backward error ||L x||_inf / (||L||_inf ||x||_inf) with the
    unmodified Liouvillian L of Eq. 3 (no trace row)."""
    Linf = np.abs(L).sum(axis=1).max()
    r = np.abs(L @ x).max()
    if Linf == 0:  # L = 0 (a single level): every x has zero backward error
        return 0.0 if r == 0 else float("inf")
    return float(r / (Linf * np.abs(x).max()))


@dataclass
class SteadyResult:
    rho: np.ndarray
    x: np.ndarray
    eta: float
    iterations: int = 0
    fill: float = 0.0
    converged: bool = True
    seconds: float = 0.0
    setup_seconds: float = 0.0


def steady_state_dense(p: Params, trace_mode: str = "replace", nth_floor: float = 1e-15) -> SteadyResult:
    """Dense LU solve of Eq. 5 (small sizes only)."""
    t0 = time.perf_counter()
    Lt, b, w, L = augmented(p, trace_mode, nth_floor)
    x = np.linalg.solve(Lt.toarray(), b)
    n = p.Nc * p.Nm
    x = trace_normalise(x, n)
    return SteadyResult(rho_from_vec(x, n), x, eta(L, x), seconds=time.perf_counter() - t0)


def steady_state_iterative(p: Params, trace_mode: str = "replace", nth_floor: float = 1e-15,
                           droptol: float = 1e-4, fill: float = 20.0, restart: int = 50,
                           rtol: float = 1e-14, max_iterations: int = 5000,
                           equilibrated: bool = False) -> SteadyResult:
    """RCM -> ILUT -> right-preconditioned GMRES(restart) on L~ (Sec. III-IV);
    equilibrated=True factors diag(r) A diag(c) (``equilibrate``) instead."""
    t0 = time.perf_counter()
    Lt, b, w, L = augmented(p, trace_mode, nth_floor)
    perm = rcm_permutation(Lt)
    A = permute_symmetric(Lt, perm)
    if equilibrated:
        r, c = equilibrate(A)
        F = ilut(sp.diags(r) @ A @ sp.diags(c), droptol, fill)
        precond = lambda v: c * F.solve(r * v)  # noqa: E731
    else:
        F = ilut(A, droptol, fill)
        precond = F.solve
    t1 = time.perf_counter()
    res = gmres_right(lambda v: A @ v, precond, b[perm], restart=restart, rtol=rtol,
                      max_iterations=max_iterations)
    x = np.empty_like(res.x)
    x[perm] = res.x
    n = p.Nc * p.Nm
    x = trace_normalise(x, n)
    t2 = time.perf_counter()
    return SteadyResult(rho_from_vec(x, n), x, eta(L, x), res.iterations,
                        F.fill_factor(A.nnz), res.converged, t2 - t0, t1 - t0)


# --------------------------------------------------------------------------
# Observables (Sec. V): <a^dag a>, <b^dag b> and the helpers used by the
# invariants of the tests.
# --------------------------------------------------------------------------

def number_operators(p: Params):
    a, b = mode_operators(p.Nc, p.Nm)
    return (a.conj().T @ a).tocsr(), (b.conj().T @ b).tocsr()


def expect(O, rho: np.ndarray) -> complex:
    """Tr(O rho)."""
    O = O.toarray() if sp.issparse(O) else np.asarray(O)
    return complex(np.trace(O @ rho))


def observables(p: Params, rho: np.ndarray) -> dict:
    na, nb = number_operators(p)
    return {"n_a": expect(na, rho).real, "n_b": expect(nb, rho).real}


def phonon_distribution(p: Params, rho: np.ndarray) -> np.ndarray:
    """P(m) = <m| Tr_cavity(rho) |m>, the phonon number distribution of Fig. 5:
    the reduced mechanical state Tr_a(rho) written out with the tensor order of
    Sec. III (h = c N_m + m) by summing the cavity blocks."""
    n = p.Nc * p.Nm
    r = np.asarray(rho).reshape(p.Nc, p.Nm, p.Nc, p.Nm)
    rho_m = np.einsum("cmcl->ml", r)  # partial trace over the cavity
    assert rho_m.shape == (p.Nm, p.Nm) and n == p.Nc * p.Nm
    return np.real(np.diag(rho_m))


def fano_factor(P: np.ndarray) -> float:
    """F = <(Delta N_b)^2> / <N_b> of a phonon distribution (Sec. V)."""
    m = np.arange(len(P), dtype=np.float64)
    mean = float(np.dot(m, P))
    var = float(np.dot(m * m, P)) - mean * mean
    return var / mean


# --------------------------------------------------------------------------
# Adjoint gradient of F(rho) for parameters theta in (Delta, E, g0, kappa).
#
# x solves A x = w e0 with A = L~ (Eq. 5).  The solution does not depend on w
# (Tr x = 1 either way), so with w held fixed dx/dtheta = -A^{-1} (dA/dtheta) x,
# where dA/dtheta is dL/dtheta in the rows of L and 0 in a replaced trace row.
# For a real loss with PyTorch-convention gradient G = dF/dRe(x) + i dF/dIm(x),
# dF/dtheta = Re(G^H dx/dtheta) = -Re(mu^H (dA/dtheta) x), A^H mu = G.
# --------------------------------------------------------------------------

THETAS = ("Delta", "E", "g0", "kappa")


def dliouvillian(p: Params, theta: str) -> sp.csr_matrix:
    """dL/dtheta from Eq. 1 and Eq. 3 (Kronecker form, column stacking)."""
    n = p.Nc * p.Nm
    I = sp.identity(n, dtype=np.complex128, format="csr")
    a, b = mode_operators(p.Nc, p.Nm)
    ad, bd = a.conj().T, b.conj().T
    num_a = ad @ a
    if theta == "kappa":
        OdO = num_a
        return sp.csr_matrix(sp.kron(a.conj(), a) - 0.5 * sp.kron(I, OdO) - 0.5 * sp.kron(OdO.T, I))
    dH = {"Delta": -num_a, "E": a + ad, "g0": (b + bd) @ num_a}[theta]
    return sp.csr_matrix(-1j * (sp.kron(I, dH) - sp.kron(dH.T, I)))


def daugmented(p: Params, theta: str, trace_mode: str = "replace") -> sp.csr_matrix:
    dL = dliouvillian(p, theta).tolil()
    if trace_mode == "replace":
        dL[0, :] = 0.0
    return sp.csr_matrix(dL)


def adjoint_gradient_dense(p: Params, G: np.ndarray, trace_mode: str = "replace",
                           nth_floor: float = 1e-15) -> dict:
    """-Re(mu^H dA/dtheta x) for each theta, with dense LU solves (small sizes)."""
    Lt, b, w, L = augmented(p, trace_mode, nth_floor)
    Ad = Lt.toarray()
    x = np.linalg.solve(Ad, b)
    x = trace_normalise(x, p.Nc * p.Nm)
    mu = np.linalg.solve(Ad.conj().T, G)
    return {t: float(-np.real(np.vdot(mu, daugmented(p, t, trace_mode) @ x))) for t in THETAS}


def adjoint_gradient_iterative(p: Params, G: np.ndarray, trace_mode: str = "replace",
                               nth_floor: float = 1e-15, droptol: float = 1e-4,
                               fill: float = 20.0, restart: int = 50, rtol: float = 1e-14) -> dict:
    """Same gradient with the paper's iterative pipeline for both solves; the
    adjoint solve uses GMRES on A^H with the preconditioner (L U)^H."""
    Lt, b, w, L = augmented(p, trace_mode, nth_floor)
    perm = rcm_permutation(Lt)
    A = permute_symmetric(Lt, perm)
    F = ilut(A, droptol, fill)
    fwd = gmres_right(lambda v: A @ v, F.solve, b[perm], restart=restart, rtol=rtol)
    AH = A.conj().T.tocsr()
    adj = gmres_right(lambda v: AH @ v, F.solve_h, np.asarray(G)[perm], restart=restart, rtol=rtol)
    x = np.empty_like(fwd.x)
    x[perm] = fwd.x
    x = trace_normalise(x, p.Nc * p.Nm)
    mu = np.empty_like(adj.x)
    mu[perm] = adj.x
    return {t: float(-np.real(np.vdot(mu, daugmented(p, t, trace_mode) @ x))) for t in THETAS}


def observable_vec(p: Params, which: str) -> np.ndarray:
    """vec(O) (Eq. 4) for O = a^dag a ('n_a') or b^dag b ('n_b')."""
    na, nb = number_operators(p)
    O = {"n_a": na, "n_b": nb}[which].toarray()
    return O.reshape(-1, order="F").astype(np.complex128)


def steady_observable(p: Params, which: str, trace_mode: str = "replace",
                      nth_floor: float = 1e-15) -> float:
    r = steady_state_dense(p, trace_mode, nth_floor)
    return observables(p, r.rho)[which]
