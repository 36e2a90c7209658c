"""Oracle: the optomechanical Liouvillian written out from its definition.

Test infrastructure only (see ``oracle/__init__.py``).

* Hamiltonian, Eq. 1 (pump frame):
  H = -Delta a^dag a + omega_m b^dag b + g0 (b + b^dag) a^dag a + E (a + a^dag),
  with Gamma_m = omega_m / Q_m.
* The variants named in Sec. VI (the conclusion) add, with X = b + b^dag,
  a quadratic ("membrane in the middle") coupling g2 X^2 a^dag a and an
  anharmonic oscillator term lam X^4; the paper prints neither coefficient,
  so g2 and lam are named here.  X^2 and X^4 are the powers of the truncated
  matrix X (the operator algebra done inside the N_m-level space), which
  differ from the infinite-space operators only in the last levels.
* Tensor order, Sec. III: a = a (x) I_b and b = I_a (x) b, so the Hilbert index
  of |c, m> is h = c * N_m + m and the dimension is n = N_c * N_m.
* Lindblad form, Eq. 3:
  L rho = -i[H, rho] + kappa D[a] rho + Gamma_m (1 + n_th) D[b] rho
          + Gamma_m n_th D[b^dag] rho,
  D[O] rho = (2 O rho O^dag - rho O^dag O - O^dag O rho) / 2.
* Column-stacked vectorisation, Eq. 4: vec(A X B) = (B^T (x) A) vec(X), so the
  vec index of rho_ij is k = i + j * n.
* Trace augmentation, Eq. 5: L~ = L + w T, T having ones in row 0 at the
  columns k = i (n + 1) of the diagonal elements, right-hand side (w, 0, ...).
  w is the mean of the diagonal of L (Sec. IV).  Two trace modes: "add" (Eq. 5
  as printed) and "replace" (row 0 of L~ is w T's row alone).
* Exact zeros are dropped (Sec. III: only the structure matters to the
  reordering; zeros arise at c = 0 in the g0 term and at truncation edges).
* n_th = 0 is replaced by a structural floor (default 1e-15) when asked
  (Sec. IV: the floor keeps the thermal entries in the structure and leaves
  the solution numerically unchanged).

Every operator is built with scipy.sparse Kronecker products, the textbook
route, so that a reader can check each term against Eq. 1, 3 and 4.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass(frozen=True)
class Params:
    """Parameters of Eq. 1 and Eq. 3 plus the Fock truncations of Sec. III."""
    Nc: int
    Nm: int
    omega_m: float = 1.0
    Delta: float = -1.0
    kappa: float = 0.5
    g0: float = 0.3
    E: float = 0.2
    Q_m: float = 1e3
    n_th: float = 0.5
    g2: float = 0.0   # quadratic coupling g2 (b + b^dag)^2 a^dag a (Sec. VI)
    lam: float = 0.0  # anharmonic term lam (b + b^dag)^4 (Sec. VI)


def lowering(N: int) -> sp.csr_matrix:
    """Truncated annihilation operator: <k-1| a |k> = sqrt(k)."""
    return sp.diags(np.sqrt(np.arange(1, N, dtype=np.float64)), 1, shape=(N, N),
                    format="csr", dtype=np.complex128)


def mode_operators(Nc: int, Nm: int):
    """a = a (x) I_b, b = I_a (x) b (Sec. III operator ordering)."""
    a = sp.kron(lowering(Nc), sp.identity(Nm, dtype=np.complex128), format="csr")
    b = sp.kron(sp.identity(Nc, dtype=np.complex128), lowering(Nm), format="csr")
    return a, b


def effective_nth(p: Params, nth_floor: float) -> float:
    return nth_floor if (p.n_th == 0.0 and nth_floor > 0.0) else p.n_th


def hamiltonian(p: Params) -> sp.csr_matrix:
    """Eq. 1 (units of hbar)."""
    a, b = mode_operators(p.Nc, p.Nm)
    ad, bd = a.conj().T, b.conj().T
    num_a = ad @ a
    X = b + bd
    H = (-p.Delta * num_a + p.omega_m * (bd @ b)
         + p.g0 * (X @ num_a) + p.E * (a + ad))
    if p.g2 != 0.0:
        H = H + p.g2 * (X @ X @ num_a)
    if p.lam != 0.0:
        H = H + p.lam * (X @ X @ X @ X)
    H = sp.csr_matrix(H)
    H.eliminate_zeros()
    return H


def collapse_terms(p: Params, nth_floor: float = 0.0):
    """(rate, operator) pairs of Eq. 3."""
    a, b = mode_operators(p.Nc, p.Nm)
    Gm = p.omega_m / p.Q_m
    nth = effective_nth(p, nth_floor)
    return [(p.kappa, a), (Gm * (1.0 + nth), b), (Gm * nth, b.conj().T.tocsr())]


def liouvillian(p: Params, nth_floor: float = 0.0) -> sp.csr_matrix:
    """Matrix of Eq. 3 in the column-stacked basis of Eq. 4 (no trace row)."""
    n = p.Nc * p.Nm
    I = sp.identity(n, dtype=np.complex128, format="csr")
    H = hamiltonian(p)
    # -i[H, rho] -> -i (I (x) H - H^T (x) I)
    L = -1j * (sp.kron(I, H) - sp.kron(H.T, I))
    for rate, O in collapse_terms(p, nth_floor):
        if rate == 0.0:
            continue
        OdO = O.conj().T @ O
        # O rho O^dag -> conj(O) (x) O ; O^dag O rho -> I (x) O^dag O ; rho O^dag O -> (O^dag O)^T (x) I
        L = L + rate * (sp.kron(O.conj(), O) - 0.5 * sp.kron(I, OdO) - 0.5 * sp.kron(OdO.T, I))
    L = sp.csr_matrix(L)
    L.eliminate_zeros()
    L.sort_indices()
    return L


def diagonal_positions(n: int) -> np.ndarray:
    """vec indices k = i (n + 1) of the diagonal elements rho_ii (Eq. 5)."""
    return np.arange(n, dtype=np.int64) * (n + 1)


def trace_weight(L: sp.csr_matrix) -> float:
    """w of Eq. 5: the mean of the diagonal of L (Sec. IV); its imaginary part
    vanishes in exact arithmetic, so the real part is taken.  w only scales
    the trace row; for a single level (n = 1) L = 0 and the mean is 0, so
    w = 1 is taken there (any nonzero w gives rho = 1)."""
    w = float(np.real(L.diagonal().sum()) / L.shape[0])
    return w if w != 0.0 else 1.0


def augmented(p: Params, trace_mode: str = "replace", nth_floor: float = 1e-15):
    """L~ of Eq. 5 and its right-hand side.

    Returns (Lt, b, w, L) with Lt CSR (sorted, exact zeros dropped)."""
    if trace_mode not in ("replace", "add"):
        raise ValueError(trace_mode)
    L = liouvillian(p, nth_floor)
    N = L.shape[0]
    n = p.Nc * p.Nm
    w = trace_weight(L)
    T = sp.csr_matrix((np.ones(n), (np.zeros(n, dtype=np.int64), diagonal_positions(n))),
                      shape=(N, N), dtype=np.complex128)
    if trace_mode == "add":
        Lt = L + w * T
    else:
        keep = sp.diags(np.r_[0.0, np.ones(N - 1)], format="csr")
        Lt = keep @ L + w * T
    Lt = sp.csr_matrix(Lt)
    Lt.eliminate_zeros()
    Lt.sort_indices()
    b = np.zeros(N, dtype=np.complex128)
    b[0] = w
    return Lt, b, w, L


def superoperator_column(p: Params, k: int, nth_floor: float = 0.0) -> np.ndarray:
    """Column k of L computed by acting with Eq. 3 on the basis matrix
    E_ij (k = i + j n) with dense matrix products -- no Kronecker identity."""
    n = p.Nc * p.Nm
    i, j = k % n, k // n
    Eij = np.zeros((n, n), dtype=np.complex128)
    Eij[i, j] = 1.0
    H = hamiltonian(p).toarray()
    out = -1j * (H @ Eij - Eij @ H)
    for rate, O in collapse_terms(p, nth_floor):
        Od = O.toarray()
        OdO = Od.conj().T @ Od
        out += rate * (Od @ Eij @ Od.conj().T - 0.5 * (Eij @ OdO + OdO @ Eij))
    return out.reshape(-1, order="F")


def liouvillian_row(p: Params, k: int, nth_floor: float = 0.0):
    """Row k of L (no trace row) from the Kronecker form, computed on its own
    so that single rows of very large Liouvillians can be checked.

    Row k = i + j n of kron(X, Y) is X[j, :] (x) Y[i, :]."""
    n = p.Nc * p.Nm
    i, j = k % n, k // n
    I = sp.identity(n, dtype=np.complex128, format="csr")
    H = hamiltonian(p)
    acc = {}

    def add_kron_row(X, Y, coef):
        xr = X.getrow(j).tocoo()
        yr = Y.getrow(i).tocoo()
        for cx, vx in zip(xr.col, xr.data):
            for cy, vy in zip(yr.col, yr.data):
                col = int(cx) * n + int(cy)
                acc[col] = acc.get(col, 0.0) + coef * vx * vy

    add_kron_row(I, H, -1j)
    add_kron_row(H.T.tocsr(), I, 1j)
    for rate, O in collapse_terms(p, nth_floor):
        if rate == 0.0:
            continue
        OdO = (O.conj().T @ O).tocsr()
        add_kron_row(O.conj().tocsr(), O, rate)
        add_kron_row(I, OdO, -0.5 * rate)
        add_kron_row(OdO.T.tocsr(), I, -0.5 * rate)
    cols = np.array(sorted(c for c, v in acc.items() if v != 0), dtype=np.int64)
    vals = np.array([acc[c] for c in cols], dtype=np.complex128)
    return cols, vals


def symmetric_pattern(A: sp.csr_matrix) -> sp.csr_matrix:
    """Structure of A + A^T (Sec. III): a pattern union, never a numeric sum."""
    P = sp.csr_matrix((np.ones(A.nnz), A.indices, A.indptr), shape=A.shape)
    S = (P + P.T).tocsr()
    S.data[:] = 1.0
    S.sort_indices()
    return S


def bandwidth_profile(A: sp.csr_matrix):
    """ub, lb, B = ub + lb + 1, up, lp, P = up + lp (Sec. II).

    up sums, over rows i, max_{a_ij != 0} (j - i); lp sums, over columns j,
    max_{a_ij != 0} (i - j).  A row or column with no entry on the relevant
    side of the diagonal contributes 0."""
    C = A.tocoo()
    r, c = C.row.astype(np.int64), C.col.astype(np.int64)
    N = A.shape[0]
    ub = int(max(0, (c - r).max())) if C.nnz else 0
    lb = int(max(0, (r - c).max())) if C.nnz else 0
    upper = np.zeros(N, dtype=np.int64)
    np.maximum.at(upper, r, c - r)
    lower = np.zeros(N, dtype=np.int64)
    np.maximum.at(lower, c, r - c)
    up, lp = int(upper.sum()), int(lower.sum())
    return dict(ub=ub, lb=lb, B=ub + lb + 1, up=up, lp=lp, P=up + lp)
