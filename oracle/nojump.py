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
  of K, then a triangular Sylvester solve by block recursion,
  ``triangular_sylvester``), or with K^dag X + X K = Y for the adjoint S^H;
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


def triangular_sylvester(T1: np.ndarray, T2: np.ndarray, Y: np.ndarray, base: int = 256) -> np.ndarray:
    """X with T1 X + X T2^dag = Y for upper triangular T1 (m x m), T2 (n x n).

    Block recursion (the Bartels-Stewart back substitution by blocks): with
    T1 = [[A, B], [0, C]] the bottom block row solves C X2 + X2 T2^dag = Y2 and
    then A X1 + X1 T2^dag = Y1 - B X2; with T2 = [[D, E], [0, F]] the right
    block column solves T1 X2 + X2 F^dag = Y2 and then T1 X1 + X1 D^dag =
    Y1 - X2 E^dag.  Blocks of at most `base` rows and columns go to LAPACK's
    ztrsyl."""
    m, n = Y.shape
    if m <= base and n <= base:
        X, scale, info = sla.lapack.ztrsyl(T1, T2, Y, trana="N", tranb="C", isgn=1)
        if info < 0:
            raise ValueError(f"ztrsyl argument {-info}")
        return X / scale
    if m >= n:
        h = m // 2
        X2 = triangular_sylvester(T1[h:, h:], T2, Y[h:], base)
        X1 = triangular_sylvester(T1[:h, :h], T2, Y[:h] - T1[:h, h:] @ X2, base)
        return np.vstack([X1, X2])
    h = n // 2
    X2 = triangular_sylvester(T1, T2[h:, h:], Y[:, h:], base)
    X1 = triangular_sylvester(T1, T2[:h, :h], Y[:, :h] - X2 @ T2[:h, h:].conj().T, base)
    return np.hstack([X1, X2])


class NoJumpInverse:
    """S^{-1} and S^{-H} by the Bartels-Stewart method: the complex Schur form
    K = Q T Q^dag is computed once; then K X + X K^dag = Y becomes
    T X' + X' T^dag = Q^dag Y Q (a triangular Sylvester equation, solved by
    ``triangular_sylvester``) with X = Q X' Q^dag.  The adjoint
    K^dag X + X K = Y becomes T^dag X' + X' T = Q^dag Y Q, brought to the same
    upper triangular form by reversing the order of rows and columns."""

    def __init__(self, p: Params, nth_floor: float = 1e-15, K: np.ndarray | None = None):
        self.n = p.Nc * p.Nm
        self.K = effective_hamiltonian(p, nth_floor) if K is None else K
        self.T, self.Q = sla.schur(self.K, output="complex")

    def __call__(self, y: np.ndarray, adjoint: bool = False) -> np.ndarray:
        n, T, Q = self.n, self.T, self.Q
        Y = np.asarray(y, dtype=np.complex128).reshape((n, n), order="F")
        Yh = Q.conj().T @ Y @ Q
        if adjoint:
            # J (reversal) turns T^dag into the upper triangular U = J T^dag J,
            # and J T J = U^dag:  U X'' + X'' U^dag = J Yh J,  X' = J X'' J
            U = T.conj().T[::-1, ::-1]
            Xh = triangular_sylvester(U, U, Yh[::-1, ::-1])[::-1, ::-1]
        else:
            Xh = triangular_sylvester(T, T, Yh)
        X = Q @ Xh @ Q.conj().T
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
