"""Writes tests/golden/ccpt_5x160_reference.json: the phonon number
distribution, its first two moments and Fano factor, and seeded entries of the
steady state of the cavity-Cooper pair transistor of Sec. V (Fig. 5: N_c = 5,
N_m = 160, E = 0.45, kappa = 0.05, Delta = -2 kappa, g0 = 0.32, n_th = 20),
computed by the oracle alone: GMRES(120) on L~ (Eq. 5) right-preconditioned
by the FP64 Bartels-Stewart inverse of the no-jump operator
(oracle/nojump.py), to a relative residual of 1e-14.  Run from the
repository root:

    python tests/golden/make_ccpt_reference.py

It takes about an hour on 8 cores (some 4,900 iterations, each a triangular
Sylvester solve of order 800).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.liouvillian import Params, augmented  # noqa: E402
from oracle.nojump import steady_state_nojump  # noqa: E402
from oracle.steady import eta, fano_factor, observables, phonon_distribution, rho_from_vec  # noqa: E402
from paper_1411_4356_gb300.workloads import CCPT  # noqa: E402


def main():
    q = CCPT.params
    p = Params(q.Nc, q.Nm, q.omega_m, q.Delta, q.kappa, q.g0, q.E, q.Q_m, q.n_th)
    t0 = time.time()
    x, its, ok, secs = steady_state_nojump(p, CCPT.trace_mode, CCPT.nth_floor, restart=CCPT.restart, rtol=1e-14,
                                           max_iterations=15000)
    n = q.Nc * q.Nm
    Lt, b, w, L = augmented(p, CCPT.trace_mode, CCPT.nth_floor)
    e = eta(L, x)
    rho = rho_from_vec(x, n)
    P = phonon_distribution(p, rho)
    m = np.arange(q.Nm, dtype=np.float64)
    rng = np.random.default_rng(4356)
    ij = rng.integers(0, n, size=(256, 2))
    obs = observables(p, rho)
    out = {
        "source": "oracle.nojump.steady_state_nojump (GMRES on L~ with the FP64 Bartels-Stewart inverse of the "
                  "no-jump operator), oracle.steady.phonon_distribution and fano_factor, written by "
                  "tests/golden/make_ccpt_reference.py",
        "params": {"Nc": q.Nc, "Nm": q.Nm, "omega_m": q.omega_m, "Delta": q.Delta, "kappa": q.kappa, "g0": q.g0,
                   "E": q.E, "Q_m": q.Q_m, "n_th": q.n_th, "nth_floor": CCPT.nth_floor,
                   "trace_mode": CCPT.trace_mode},
        "eta": e, "iterations": its, "converged": bool(ok), "seconds": time.time() - t0,
        "n_a": obs["n_a"], "n_b": obs["n_b"],
        "diag_re": np.real(np.diag(rho)).tolist(), "diag_im": np.imag(np.diag(rho)).tolist(),
        "P": P.tolist(), "mean": float(m @ P), "second": float((m * m) @ P), "fano": fano_factor(P),
        "samples": [[int(i), int(j), float(rho[i, j].real), float(rho[i, j].imag)] for i, j in ij],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ccpt_5x160_reference.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(f"wrote {path}: eta {e:.2e}, {its} iterations, F {out['fano']:.4f}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
