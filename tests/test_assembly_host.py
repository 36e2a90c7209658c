"""The assembly's closed-form rows (om_liouvillian_row_host: the row function
the assembly kernels evaluate, run on the host) against the oracle's rows of
the Kronecker form of Eq. 3, on sampled rows up to the 16,000,000-row system
and with the Sec. VI variants.  No GPU needed.  Columns bit-exact; values
within 64 eps times the row's absolute sum (the oracle sums up to eight
Kronecker terms per entry)."""
import numpy as np
import pytest

from oracle.liouvillian import Params, liouvillian_row
from paper_1411_4356_gb300 import LARGE, api
from paper_1411_4356_gb300.workloads import SystemParams

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


def oparams(p):
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th, p.g2, p.lam)


@pytest.mark.parametrize("p,floor", [(SystemParams(3, 5, **BASE), 1e-15),
                                     (SystemParams(4, 12, **{**BASE, "g2": 0.05, "lam": 0.004}), 1e-15),
                                     (SystemParams(5, 9, **{**BASE, "n_th": 0.0}), 0.0),
                                     (LARGE.params, LARGE.nth_floor)],
                         ids=["3x5", "4x12-variants", "5x9-nth0", "16M"])
def test_rows_match_oracle(p, floor):
    N = p.N
    rng = np.random.default_rng(p.Nc * 1000 + p.Nm)
    ks = sorted({0, 1, p.Nm, N - 1, N // 2, *rng.integers(0, N, size=40).tolist()})
    for k in ks:
        cols, vals = api.liouvillian_row_host(p, k, floor)
        rc, rv = liouvillian_row(oparams(p), int(k), floor)
        keep = np.abs(rv) > 0
        np.testing.assert_array_equal(cols, np.asarray(rc)[keep])
        scale = max(1.0, float(np.abs(rv).sum()))
        assert np.abs(vals - np.asarray(rv)[keep]).max(initial=0.0) <= 64 * np.finfo(float).eps * scale, k
