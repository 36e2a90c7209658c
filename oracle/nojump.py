"""Oracle: the no-jump part of the Lindblad generator and its inverse.

Test infrastructure only (see ``oracle/__init__.py``).

Eq. 3 splits into a part that maps rho to K rho + rho K^dag and the jump
terms gamma_O O rho O^dag, with the effective non-Hermitian Hamiltonian

    K = -i H - (1/2) sum_O gamma_O O^dag O          (H of Eq. 1),

so that L rho = K rho + rho K^dag + sum_O gamma_O O rho O^dag.  In the column-
stacked basis of Eq. 4 (vec(A X B) = (B^T (x) A) vec(X)) the first part is the
Kronecker sum

    S = I (x) K + conj(K) (x) I .

The paper does not use S; the GPU path preconditions GMRES with S^{-1} as a
second preconditioner beside the ILUT of Sec. II.  This module writes S and
its inverse out from that definition:

* ``effective_hamiltonian`` -- K as a dense matrix, from the oracle's H and
  collapse operators (Eq. 1 and Eq. 3);
* ``nojump_operator`` -- S as a sparse matrix (Kronecker products);
* ``NoJumpInverse`` / ``nojump_solve`` -- X with K X + X K^dag = Y (a
  Sylvester equation, solved by the Bartels-Stewart method: complex Schur form
  of K, then a triangular Sylvester solve), or with K^dag X + X K = Y for the
  adjoint S^H;
* ``nojump_solve_dense`` -- the same by dense LU of S (tiny sizes only);
* ``steady_state_nojump`` -- GMRES on L~ (Eq. 5) right-preconditioned by
  S^{-1}; its answer is the steady state of Eq. 5 whatever the
  preconditioner.
"""
from __future__ import annotations

import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .gmres import gmres_right
from .liouvillian import Params, augmented, collapse_terms, hamiltonian


def effective_hamiltonian(p: Params, nth_floor: float = 1e-15) -> np.ndarray:
    """K = -i H - 1/2 sum_O gamma_O O^dag O (dense n x n, complex128)."""
    K = -1j * hamiltonian(p).toarray()
    for rate, O in collapse_terms(p, nth_floor):
        Od = O.toarray()
        K -= 0.5 * rate * (Od.conj().T @ Od)
    return K


def nojump_operator(p: Params, nth_floor: float = 1e-15) -> sp.csr_matrix:
    """S = I (x) K + conj(K) (x) I, the matrix of rho -> K rho + rho K^dag."""
    K = sp.csr_matrix(effective_hamiltonian(p, nth_floor))
    n = K.shape[0]
    I = sp.identity(n, dtype=np.complex128, format="csr")
    S = sp.csr_matrix(sp.kron(I, K) + sp.kron(K.conj(), I))
    S.eliminate_zeros()
    S.sort_indices()
    return S


def jump_operator(p: Params, nth_floor: float = 1e-15) -> sp.csr_matrix:
    """J = sum_O gamma_O conj(O) (x) O, the matrix of the jump terms O rho O^dag."""
    n = p.Nc * p.Nm
    J = sp.csr_matrix((n * n, n * n), dtype=np.complex128)
    for rate, O in collapse_terms(p, nth_floor):
        if rate != 0.0:
            J = J + rate * sp.kron(O.conj(), O)
    J = sp.csr_matrix(J)
    J.eliminate_zeros()
    return J


class NoJumpInverse:
    """S^{-1} and S^{-H} by the Bartels-Stewart method: the complex Schur form
    K = Q T Q^dag is computed once; then K X + X K^dag = Y becomes
    T X' + X' T^dag = Q^dag Y Q (a triangular Sylvester equation, LAPACK
    ztrsyl) with X = Q X' Q^dag."""

    def __init__(self, p: Params, nth_floor: float = 1e-15, K: np.ndarray | None = None):
        self.n = p.Nc * p.Nm
        self.K = effective_hamiltonian(p, nth_floor) if K is None else K
        self.T, self.Q = sla.schur(self.K, output="complex")

    def __call__(self, y: np.ndarray, adjoint: bool = False) -> np.ndarray:
        n, T, Q = self.n, self.T, self.Q
        Y = np.asarray(y, dtype=np.complex128).reshape((n, n), order="F")
        Yh = Q.conj().T @ Y @ Q
        # forward: T X' + X' T^dag = Yh;  adjoint (K^dag X + X K = Y): T^dag X' + X' T = Yh
        trana, tranb = ("C", "N") if adjoint else ("N", "C")
        Xh, scale, info = sla.lapack.ztrsyl(T, T, Yh, trana=trana, tranb=tranb, isgn=1)
        if info < 0:
            raise ValueError(f"ztrsyl argument {-info}")
        X = Q @ (Xh / scale) @ Q.conj().T
        return X.reshape(-1, order="F")


def nojump_solve(p: Params, y: np.ndarray, nth_floor: float = 1e-15, adjoint: bool = False,
                 K: np.ndarray | None = None) -> np.ndarray:
    """vec(X) with K X + X K^dag = Y (adjoint: K^dag X + X K = Y), Y = unvec(y)."""
    return NoJumpInverse(p, nth_floor, K)(y, adjoint)


def nojump_solve_dense(p: Params, y: np.ndarray, nth_floor: float = 1e-15, adjoint: bool = False) -> np.ndarray:
    """The same solve by dense LU of the n^2 x n^2 matrix S (tiny sizes only)."""
    S = nojump_operator(p, nth_floor).toarray()
    if adjoint:
        S = S.conj().T
    return np.linalg.solve(S, np.asarray(y, dtype=np.complex128))


def steady_state_nojump(p: Params, trace_mode: str = "replace", nth_floor: float = 1e-15, restart: int = 50,
                        rtol: float = 1e-14, max_iterations: int = 2000):
    """GMRES(restart) on L~ x = (w, 0, ...)^T in natural order, right-preconditioned
    by S^{-1}; returns (x normalised to unit trace, iterations, converged, seconds)."""
    from .steady import trace_normalise

    t0 = time.perf_counter()
    Lt, b, w, L = augmented(p, trace_mode, nth_floor)
    Sinv = NoJumpInverse(p, nth_floor)
    res = gmres_right(lambda v: Lt @ v, Sinv, b, restart=restart, rtol=rtol, max_iterations=max_iterations)
    x = trace_normalise(res.x, p.Nc * p.Nm)
    return x, res.iterations, res.converged, time.perf_counter() - t0
