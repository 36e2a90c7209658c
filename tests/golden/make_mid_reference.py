"""Writes tests/golden/mid_10x60_reference.json: sampled entries of the steady
state of the 360,000-row system (N_c = 10, N_m = 60), computed by the oracle
alone (RCM, ILUT(1e-5, 100), right-preconditioned GMRES(50) to a relative
residual of 1e-15; Sec. III-IV), for the full-size parity test of the GPU
path.  Run from the repository root:

    python tests/golden/make_mid_reference.py

It takes about twenty minutes on one core (the ILUT dominates).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.liouvillian import Params  # noqa: E402
from oracle.steady import observables, steady_state_iterative  # noqa: E402
from paper_1411_4356_gb300.workloads import MID  # noqa: E402


def main():
    q = MID.params
    p = Params(q.Nc, q.Nm, q.omega_m, q.Delta, q.kappa, q.g0, q.E, q.Q_m, q.n_th)
    t0 = time.time()
    r = steady_state_iterative(p, MID.trace_mode, MID.nth_floor, droptol=MID.droptol, fill=MID.fill,
                               restart=MID.restart, rtol=1e-15, max_iterations=3000)
    rho = r.rho
    n = q.Nc * q.Nm
    rng = np.random.default_rng(4356)
    ij = rng.integers(0, n, size=(256, 2))
    obs = observables(p, rho)
    out = {
        "source": "oracle.steady.steady_state_iterative (RCM, ILUT, GMRES; Sec. III-IV), written by "
                  "tests/golden/make_mid_reference.py",
        "params": {"Nc": q.Nc, "Nm": q.Nm, "omega_m": q.omega_m, "Delta": q.Delta, "kappa": q.kappa, "g0": q.g0,
                   "E": q.E, "Q_m": q.Q_m, "n_th": q.n_th, "trace_mode": MID.trace_mode, "nth_floor": MID.nth_floor},
        "solver": {"droptol": MID.droptol, "fill": MID.fill, "restart": MID.restart, "rtol": 1e-15,
                   "iterations": int(r.iterations), "converged": bool(r.converged), "eta": float(r.eta),
                   "seconds": time.time() - t0},
        "diag_re": [float(x) for x in np.real(np.diag(rho))],
        "diag_im": [float(x) for x in np.imag(np.diag(rho))],
        "samples": [[int(i), int(j), float(rho[i, j].real), float(rho[i, j].imag)] for i, j in ij],
        "n_a": float(obs["n_a"]),
        "n_b": float(obs["n_b"]),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mid_10x60_reference.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, out["solver"])


if __name__ == "__main__":
    main()
