"""Oracle wrappers for the reordering (Sec. III) and the incomplete LU
factorisation (Sec. II) implemented in plain C in ``oracle_native.c``.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import native
from .liouvillian import symmetric_pattern

_I64P = native._I64P
_I32P = native._I32P
_F64P = native._F64P


def rcm_permutation(A: sp.csr_matrix) -> np.ndarray:
    """RCM order of the structure of A + A^T (Sec. III); perm[new] = old."""
    S = symmetric_pattern(A)
    ptr = np.ascontiguousarray(S.indptr, dtype=np.int64)
    idx = np.ascontiguousarray(S.indices, dtype=np.int32)
    perm = np.empty(S.shape[0], dtype=np.int32)
    rc = native.lib().oracle_rcm(S.shape[0], native.ptr(ptr, _I64P), native.ptr(idx, _I32P),
                                 native.ptr(perm, _I32P))
    if rc != 0:
        raise MemoryError("oracle_rcm")
    return perm


def permute_symmetric(A: sp.csr_matrix, perm: np.ndarray) -> sp.csr_matrix:
    """A_rcm = P A P^T: A_rcm[r, c] = A[perm[r], perm[c]] (Sec. III applies the
    same order to rows and columns)."""
    B = A[perm][:, perm].tocsr()
    B.sort_indices()
    return B


def equilibrate(A: sp.csr_matrix):
    """Row and column scalings (r, c) of the equilibration step that the
    iLUTP of Sec. II performs as SuperLU runs it, before it factors: r_i =
    1 / max_j |a_ij|, then c_j = 1 / max_i |r_i a_ij|, so that every row of
    diag(r) A and every column of diag(r) A diag(c) has largest modulus 1 (a
    row of the latter has largest modulus >= 1).  A row or column without
    entries keeps the scale 1.  The factors are then those of
    diag(r) A diag(c), and the preconditioner is M^{-1} = diag(c) (L U)^{-1}
    diag(r)."""
    A = sp.csr_matrix(A)
    absA = abs(A)
    rmax = absA.max(axis=1).toarray().ravel()
    r = np.where(rmax > 0, 1.0 / np.where(rmax > 0, rmax, 1.0), 1.0)
    cmax = (sp.diags(r) @ absA).max(axis=0).toarray().ravel()
    c = np.where(cmax > 0, 1.0 / np.where(cmax > 0, cmax, 1.0), 1.0)
    return r, c


@dataclass
class ILUFactors:
    n: int
    lp: np.ndarray
    li: np.ndarray
    lx: np.ndarray
    up: np.ndarray
    ui: np.ndarray
    ux: np.ndarray
    n_guarded: int
    q: np.ndarray | None = None  # ILUTP: q[k] = column at position k (A Q ~ L U)
    n_swaps: int = 0

    @property
    def nnz_l(self) -> int:
        return int(self.lp[-1])

    @property
    def nnz_u(self) -> int:
        return int(self.up[-1])

    def fill_factor(self, nnz_a: int) -> float:
        """(NNZ(L) + NNZ(U)) / NNZ(A) (Sec. IV), L counted without its unit diagonal."""
        return (self.nnz_l + self.nnz_u) / nnz_a

    def L(self) -> sp.csr_matrix:
        """Unit lower factor with its diagonal, as a scipy matrix."""
        S = sp.csr_matrix((self.lx, self.li, self.lp), shape=(self.n, self.n))
        return (S + sp.identity(self.n, dtype=np.complex128)).tocsr()

    def U(self) -> sp.csr_matrix:
        U = sp.csr_matrix((self.ux, self.ui, self.up), shape=(self.n, self.n))
        U.sort_indices()
        return U

    # M^{-1} v and M^{-H} v with M = L U (the preconditioner of Eq. 6), or
    # M = L U Q^T with column pivoting: M^{-1} = Q U^{-1} L^{-1},
    # M^{-H} = L^{-H} U^{-H} Q^T
    def solve(self, v: np.ndarray) -> np.ndarray:
        x = self._solve(v)
        if self.q is not None:
            out = np.empty_like(x)
            out[self.q] = x
            return out
        return x

    def solve_h(self, v: np.ndarray) -> np.ndarray:
        """M^{-H} v."""
        v = np.asarray(v, dtype=np.complex128)
        if self.q is not None:
            v = v[self.q]
        return self._solve_h(v)

    def _solve(self, v: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(v, dtype=np.complex128).copy()
        Lb = native.lib()
        xp = x.view(np.float64).ctypes.data_as(_F64P)
        Lb.oracle_lsolve(self.n, native.ptr(self.lp, _I64P), native.ptr(self.li, _I32P),
                         self.lx.view(np.float64).ctypes.data_as(_F64P), xp, xp)
        Lb.oracle_usolve(self.n, native.ptr(self.up, _I64P), native.ptr(self.ui, _I32P),
                         self.ux.view(np.float64).ctypes.data_as(_F64P), xp, xp)
        return x

    def _solve_h(self, v: np.ndarray) -> np.ndarray:
        """(L U)^{-H} v = L^{-H} U^{-H} v."""
        x = np.ascontiguousarray(v, dtype=np.complex128).copy()
        Lb = native.lib()
        xp = x.view(np.float64).ctypes.data_as(_F64P)
        Lb.oracle_uhsolve(self.n, native.ptr(self.up, _I64P), native.ptr(self.ui, _I32P),
                          self.ux.view(np.float64).ctypes.data_as(_F64P), xp, xp)
        Lb.oracle_lhsolve(self.n, native.ptr(self.lp, _I64P), native.ptr(self.li, _I32P),
                          self.lx.view(np.float64).ctypes.data_as(_F64P), xp, xp)
        return x


def ilut(A: sp.csr_matrix, droptol: float, fill: float, cap: str = "row") -> ILUFactors:
    """ILUT(d, p) of A (rows sorted by column); see oracle_native.c for the
    dropping rules read from Sec. II and Sec. IV.  cap="row": at most
    floor(p nnz_i / 2) entries in each of the L and U parts of row i;
    cap="total": NNZ(L) + NNZ(U) <= p NNZ(A) as a running budget over the rows
    (oracle_ilut_total)."""
    if cap not in ("row", "total"):
        raise ValueError(cap)
    A = sp.csr_matrix(A)
    A.sort_indices()
    n = A.shape[0]
    ap = np.ascontiguousarray(A.indptr, dtype=np.int64)
    ai = np.ascontiguousarray(A.indices, dtype=np.int32)
    ax = np.ascontiguousarray(A.data, dtype=np.complex128)
    nnz_row = np.diff(ap)
    if cap == "row":
        cap_row = np.maximum(np.floor(fill * nnz_row / 2.0).astype(np.int64), 1)
        size = int(cap_row.sum()) + n
    else:
        size = int(np.floor(fill * float(ap[-1]))) + n
    lp = np.zeros(n + 1, dtype=np.int64)
    up = np.zeros(n + 1, dtype=np.int64)
    li = np.zeros(size, dtype=np.int32)
    ui = np.zeros(size, dtype=np.int32)
    lx = np.zeros(size, dtype=np.complex128)
    ux = np.zeros(size, dtype=np.complex128)
    ng = np.zeros(1, dtype=np.int64)
    fn = native.lib().oracle_ilut if cap == "row" else native.lib().oracle_ilut_total
    rc = fn(
        n, native.ptr(ap, _I64P), native.ptr(ai, _I32P), ax.view(np.float64).ctypes.data_as(_F64P),
        float(droptol), float(fill),
        size, native.ptr(lp, _I64P), native.ptr(li, _I32P), lx.view(np.float64).ctypes.data_as(_F64P),
        size, native.ptr(up, _I64P), native.ptr(ui, _I32P), ux.view(np.float64).ctypes.data_as(_F64P),
        native.ptr(ng, _I64P))
    if rc != 0:
        raise RuntimeError(f"oracle_ilut failed ({rc})")
    nl, nu = int(lp[-1]), int(up[-1])
    return ILUFactors(n, lp, li[:nl].copy(), lx[:nl].copy(), up, ui[:nu].copy(), ux[:nu].copy(),
                      int(ng[0]))


def ilutp(A: sp.csr_matrix, droptol: float, fill: float, permtol: float) -> ILUFactors:
    """ILUTP(d, p, permtol): ILUT with threshold column pivoting (the iLUTP of
    Sec. II); see oracle_ilutp in oracle_native.c.  The factors satisfy
    A Q ~ L U and solve() applies M^{-1} = Q U^{-1} L^{-1}."""
    A = sp.csr_matrix(A)
    A.sort_indices()
    n = A.shape[0]
    ap = np.ascontiguousarray(A.indptr, dtype=np.int64)
    ai = np.ascontiguousarray(A.indices, dtype=np.int32)
    ax = np.ascontiguousarray(A.data, dtype=np.complex128)
    nnz_row = np.diff(ap)
    cap_row = np.maximum(np.floor(fill * nnz_row / 2.0).astype(np.int64), 1)
    cap = int(cap_row.sum()) + n
    lp = np.zeros(n + 1, dtype=np.int64)
    up = np.zeros(n + 1, dtype=np.int64)
    li = np.zeros(cap, dtype=np.int32)
    ui = np.zeros(cap, dtype=np.int32)
    lx = np.zeros(cap, dtype=np.complex128)
    ux = np.zeros(cap, dtype=np.complex128)
    q = np.zeros(max(n, 1), dtype=np.int32)
    ng = np.zeros(1, dtype=np.int64)
    ns = np.zeros(1, dtype=np.int64)
    rc = native.lib().oracle_ilutp(
        n, native.ptr(ap, _I64P), native.ptr(ai, _I32P), ax.view(np.float64).ctypes.data_as(_F64P),
        float(droptol), float(fill), float(permtol),
        cap, native.ptr(lp, _I64P), native.ptr(li, _I32P), lx.view(np.float64).ctypes.data_as(_F64P),
        cap, native.ptr(up, _I64P), native.ptr(ui, _I32P), ux.view(np.float64).ctypes.data_as(_F64P),
        native.ptr(q, _I32P), native.ptr(ng, _I64P), native.ptr(ns, _I64P))
    if rc != 0:
        raise RuntimeError(f"oracle_ilutp failed ({rc})")
    nl, nu = int(lp[-1]), int(up[-1])
    return ILUFactors(n, lp, li[:nl].copy(), lx[:nl].copy(), up, ui[:nu].copy(), ux[:nu].copy(),
                      int(ng[0]), q[:n].copy(), int(ns[0]))
