"""The reverse Cuthill-McKee order computed on the device (om_permute, and
om_permute_ex with bit 0 set), level by level, against the serial order of
the host (om_permute_ex, bit 0 clear) and the oracle's
(oracle.reorder_factor.rcm_permutation): bit-exact permutations, on connected
Liouvillians and on ones that fall apart into many components (g0 = E = 0
decouples the coherences), and the permuted matrices equal; then the host and
device orders at 360,000 and 16,000,000 rows, timed."""
import time

import numpy as np
import pytest
import torch

from oracle.liouvillian import Params, augmented
from oracle.reorder_factor import rcm_permutation
from paper_1411_4356_gb300 import LARGE, MID, api
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


def oparams(p):
    return Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th, p.g2, p.lam)


@pytest.mark.parametrize("Nc,Nm,kw", [(1, 1, {}), (2, 3, {}), (4, 8, {}), (10, 20, {}), (6, 20, dict(g2=0.05)),
                                      (4, 6, dict(g0=0.0, E=0.0)), (3, 5, dict(g0=0.0, E=0.0, n_th=0.0))])
@pytest.mark.parametrize("mode", ["replace", "add"])
def test_device_order_is_the_serial_order(Nc, Nm, kw, mode):
    p = SystemParams(Nc, Nm, **{**BASE, **kw})
    A = api.build_liouvillian(p, mode)
    Ad, perm_d = api.permute(A, device_order=True)
    Ah, perm_h = api.permute(A, device_order=False)
    assert torch.equal(perm_d, perm_h)
    Lt, *_ = augmented(oparams(p), mode, 1e-15)
    np.testing.assert_array_equal(perm_d.cpu().numpy(), rcm_permutation(Lt))
    for a, b in zip(Ad.export(), Ah.export()):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("w", [MID, LARGE], ids=["360k", "16M"])
def test_device_order_at_size(w):
    p = w.params
    A = api.build_liouvillian(p, w.trace_mode, w.nth_floor)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, perm_h = api.permute(A, device_order=False)
    t1 = time.perf_counter()
    _, perm_d = api.permute(A, device_order=True)
    t2 = time.perf_counter()
    print(f"RCM at {A.N} rows: host {t1 - t0:.3f} s, device {t2 - t1:.3f} s")
    assert torch.equal(perm_d, perm_h)
