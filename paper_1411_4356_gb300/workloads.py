"""Synthetic workloads: parameter sets shaped like the paper's systems.

Holds parameter values and the seeded draws of the batched sweep only -- no
arithmetic of the method.  Shared by the CUDA path, the tests and bench.py.
"""
from __future__ import annotations

from dataclasses import dataclass, replace


@dataclass(frozen=True)
class SystemParams:
    """Eq. 1 / Eq. 3 parameters (units of omega_m) and Fock cutoffs (Sec. III)."""
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

    def with_(self, **kw) -> "SystemParams":
        return replace(self, **kw)

    @property
    def n(self) -> int:
        return self.Nc * self.Nm

    @property
    def N(self) -> int:
        return self.n * self.n


@dataclass(frozen=True)
class Workload:
    name: str
    params: SystemParams
    droptol: float
    fill: float
    restart: int
    tol: float
    precision: int = 0
    trace_mode: str = "replace"
    nth_floor: float = 1e-15
    refill: float = 100.0  # fill cap for a factor whose stability estimate fails


# tiny: 1,600 rows, checked against dense LU
TINY = Workload("tiny_4x10", SystemParams(4, 10, 1.0, -1.0, 0.5, 0.3, 0.2, 1e3, 0.5),
                droptol=1e-4, fill=10.0, restart=30, tol=1e-12)
# mid: 360,000 rows, ~3.9M nonzeros.  The drop tolerance 1e-5 is kept; the
# fill cap is raised from 10 to 100 because ILUT capped at 10 is unstable on
# this system (the factor's inverse overflows).
MID = Workload("mid_10x60", SystemParams(10, 60, 1.0, -1.0, 0.3, 0.5, 0.3, 1e4, 1.0),
               droptol=1e-5, fill=100.0, restart=50, tol=1e-10)
# large: 16M rows, n_th = 0 floored to 1e-15 (Sec. IV), complex64 inner solves
LARGE = Workload("large_20x200", SystemParams(20, 200, 1.0, -1.0, 0.5, 1.5, 0.5, 1e4, 0.0),
                 droptol=1e-4, fill=10.0, restart=30, tol=1e-10, precision=1)
# adjoint: 1.44M rows.  ILUT with d = 1e-4 (caps 10, 30, 100) or d = 1e-5
# (cap 100) leaves an unstable factor at this size, so the gradient checks
# run on smaller systems with the 360,000-row parameters.
ADJOINT = Workload("adjoint_12x100", SystemParams(12, 100, 1.0, -1.0, 0.5, 1.0, 0.4, 1e4, 0.5),
                   droptol=1e-4, fill=10.0, restart=30, tol=1e-10)
# the paper's application (Sec. V, Fig. 5): the cavity-Cooper pair transistor
# at N_c = 5, N_m = 160 (640,000 rows), n_th = 20, Delta = -2 kappa, in the
# single-photon strong-coupling regime; Q_m is not printed for this case and
# the 1e4 of the other systems is taken.  The thermal jumps (n_th = 20) are
# strong against the no-jump part, so GMRES needs thousands of iterations and
# a restart of 120 (100 stagnates); mixed precision is used.  The slow
# mechanical mode amplifies the backward error about 2e4-fold in the entries
# of rho, so the solve goes to eta 5e-14 for rho to be within 1e-9.
CCPT = Workload("ccpt_5x160", SystemParams(5, 160, 1.0, -0.1, 0.05, 0.32, 0.45, 1e4, 20.0),
                droptol=1e-4, fill=200.0, restart=120, tol=5e-14, precision=1)
# batched sweep base parameters (N_c = 6; Delta and N_m drawn per system).
# ILUT(1e-5, 60): with caps of 20 and 40 some draws give an unstable factor.
BATCH_BASE = SystemParams(6, 20, 1.0, 0.0, 0.4, 0.8, 0.2, 1e3, 0.2)
BATCH_NM = (20, 30, 40, 60)
BATCH = Workload("batched_6xNm", BATCH_BASE, droptol=1e-5, fill=60.0, restart=30, tol=1e-10)


def batched_draws(count: int = 512, seed: int = 4356):
    """Delta ~ U[-3, 1] for all systems first, then N_m uniform over BATCH_NM."""
    import numpy as np

    rng = np.random.default_rng(seed)
    deltas = rng.uniform(-3.0, 1.0, size=count)
    nms = rng.choice(np.array(BATCH_NM), size=count)
    return [BATCH_BASE.with_(Delta=float(d), Nm=int(m)) for d, m in zip(deltas, nms)]
