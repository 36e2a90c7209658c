"""Oracle: restarted GMRES (Sec. IV) with right preconditioning.

Test infrastructure only (see ``oracle/__init__.py``).

Follows the generalized minimal residual method of Saad & Schultz (the
paper's GMRES reference, Sec. IV) in its textbook form:

  r0 = b - A x0, beta = ||r0||_2, v_1 = r0 / beta
  Arnoldi with modified Gram-Schmidt on A M^{-1}:
      w = A M^{-1} v_j ; h_ij = <v_i, w>, w -= h_ij v_i  (i = 1..j)
      h_{j+1,j} = ||w||_2 ; v_{j+1} = w / h_{j+1,j}
  Givens rotations reduce H to upper triangular form; |g_{j+1}| is the
  residual norm of the current iterate.
  At the end of a cycle y = argmin ||beta e1 - H y||, x = x0 + M^{-1} V y.
  Restart after m steps (the paper restarts after 10 steps; m is a parameter).

Right preconditioning (A M^{-1} u = b, x = M^{-1} u) solves the same system
as the left-preconditioned Eq. 6 and leaves the GMRES residual equal to the
true residual of the unpreconditioned system.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List

import numpy as np


@dataclass
class GmresResult:
    x: np.ndarray
    converged: bool
    iterations: int
    cycles: int
    residual_history: List[float] = field(default_factory=list)


def gmres_right(matvec: Callable[[np.ndarray], np.ndarray],
                precond: Callable[[np.ndarray], np.ndarray],
                b: np.ndarray, x0: np.ndarray | None = None, restart: int = 10,
                rtol: float = 1e-14, max_iterations: int = 5000) -> GmresResult:
    """Solve A x = b; stop when ||b - A x||_2 <= rtol * ||b||_2 (checked with the
    true residual at the end of each cycle)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return GmresResult(np.zeros_like(b), True, 0, 0, [0.0])
    target = rtol * bnorm
    history = []
    iterations = 0
    cycles = 0
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= target:
            return GmresResult(x, True, iterations, cycles, history)
        if iterations >= max_iterations:
            return GmresResult(x, False, iterations, cycles, history)
        cycles += 1
        m = restart
        V = np.zeros((m + 1, b.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = matvec(precond(V[j]))
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            # apply the previous rotations to column j
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            # new rotation zeroing H[j+1, j]
            a_, b_ = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a_) ** 2 + abs(b_) ** 2)
            if den == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            elif a_ == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a_) / den
                sn[j] = (a_ / abs(a_)) * np.conj(b_) / den
            H[j, j] = cs[j] * a_ + sn[j] * b_
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            iterations += 1
            if abs(g[j + 1]) <= target or H[j, j] == 0.0 or iterations >= max_iterations:
                break
        # back substitution on the k x k triangle
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + precond(V[:k].T @ y)
