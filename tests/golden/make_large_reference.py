"""Writes tests/golden/large_20x200_reference.json: sampled entries of the
steady state of the 16,000,000-row system (N_c = 20, N_m = 200, n_th = 0
floored to 1e-15 as in Sec. IV), computed by the oracle alone: GMRES on
L~ (Eq. 5) right-preconditioned by the inverse of the no-jump operator
K rho + rho K^dag, applied by the Bartels-Stewart method in FP64
(oracle/nojump.py), to a relative residual of 1e-15.  Run from the
repository root:

    python tests/golden/make_large_reference.py

It takes about an hour and some 40 GB of host memory (one triangular
Sylvester solve of order 4000 per iteration).
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
from oracle.steady import eta, observables, rho_from_vec  # noqa: E402
from paper_1411_4356_gb300.workloads import LARGE  # noqa: E402


def main():
    q = LARGE.params
    p = Params(q.Nc, q.Nm, q.omega_m, q.Delta, q.kappa, q.g0, q.E, q.Q_m, q.n_th)
    t0 = time.time()
    x, its, ok, secs = steady_state_nojump(p, LARGE.trace_mode, LARGE.nth_floor, restart=80, rtol=1e-15,
                                           max_iterations=400)
    n = q.Nc * q.Nm
    Lt, b, w, L = augmented(p, LARGE.trace_mode, LARGE.nth_floor)
    e = eta(L, x)
    del Lt, L
    rho = rho_from_vec(x, n)
    rng = np.random.default_rng(4356)
    ij = rng.integers(0, n, size=(256, 2))
    obs = observables(p, rho)
    out = {
        "source": "oracle.nojump.steady_state_nojump (GMRES on L~ with the FP64 Bartels-Stewart inverse of the "
                  "no-jump operator), written by tests/golden/make_large_reference.py",
        "params": {"Nc": q.Nc, "Nm": q.Nm, "omega_m": q.omega_m, "Delta": q.Delta, "kappa": q.kappa, "g0": q.g0,
                   "E": q.E, "Q_m": q.Q_m, "n_th": q.n_th, "nth_floor": LARGE.nth_floor,
                   "trace_mode": LARGE.trace_mode},
        "eta": e, "iterations": its, "converged": bool(ok), "seconds": time.time() - t0,
        "n_a": obs["n_a"], "n_b": obs["n_b"],
        "diag_re": np.real(np.diag(rho)).tolist(), "diag_im": np.imag(np.diag(rho)).tolist(),
        "samples": [[int(i), int(j), float(rho[i, j].real), float(rho[i, j].imag)] for i, j in ij],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large_20x200_reference.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(f"wrote {path}: eta {e:.2e}, {its} iterations, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
