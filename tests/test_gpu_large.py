"""The 16,000,000-row system (N_c = 20, N_m = 200, g0 = 1.5, n_th = 0 floored
to 1e-15 as in Sec. IV) in the launch configuration bench.py times: mixed
precision (complex64 inner GMRES with the TF32 no-jump preconditioner inside
FP64 refinement) at eta <= 1e-12, and the FP64 form.  Expected values: the
oracle's (tests/golden/large_20x200_reference.json, written by
make_large_reference.py: GMRES with the FP64 Bartels-Stewart no-jump inverse
to a relative residual of 1e-15), on the 4000 diagonal entries and 256 seeded
entries, plus properties that hold exactly at any size: unit trace,
Hermiticity and the truncated identity kappa <a^dag a> = -2 E Im<a>."""
import json
import os

import numpy as np
import pytest
import torch

from paper_1411_4356_gb300 import LARGE, api

pytestmark = pytest.mark.gpu

PATH = os.path.join(os.path.dirname(__file__), "golden", "large_20x200_reference.json")


@pytest.fixture(scope="module")
def system():
    A = api.build_liouvillian(LARGE.params, LARGE.trace_mode, LARGE.nth_floor)
    M = api.nojump_factor(LARGE.params, nth_floor=LARGE.nth_floor, eig32=True)
    return A, M


def invariants(rho, p):
    r = rho
    n = p.Nc * p.Nm
    tr = complex(torch.diagonal(r).sum().item())
    herm = float((r - r.conj().t()).abs().max().item())
    c = torch.arange(n, device=r.device) // p.Nm
    na = float((torch.diagonal(r).real * c).sum().item())
    h = torch.arange(n - p.Nm, device=r.device)
    a_exp = complex((torch.sqrt((h // p.Nm + 1).double()) * r[h + p.Nm, h]).sum().item())
    return abs(tr - 1), herm, abs(p.kappa * na + 2 * p.E * a_exp.imag)


@pytest.mark.parametrize("precision", [1, 0])
def test_16M_rows(system, precision):
    A, M = system
    rho, info = api.steady_state_solve_nojump(A, M, restart=50, tol=1e-12, precision=precision)
    assert info.status == 0 and info.eta <= 1e-12
    tr, herm, ident = invariants(rho, LARGE.params)
    print(f"precision {precision}: {info.iterations} iterations, eta {info.eta:.1e}, "
          f"|Tr-1| {tr:.1e}, herm {herm:.1e}, identity {ident:.1e}")
    assert tr <= 1e-12 and herm <= 1e-9 and ident <= 1e-10
    if not os.path.exists(PATH):
        pytest.skip("no stored oracle reference at 16M rows")
    ref = json.load(open(PATH))
    diag = np.array(ref["diag_re"]) + 1j * np.array(ref["diag_im"])
    got = torch.diagonal(rho).cpu().numpy()
    assert np.abs(got - diag).max() <= 1e-9
    s = np.array(ref["samples"])
    i = torch.from_numpy(s[:, 0].astype(np.int64)).cuda()
    j = torch.from_numpy(s[:, 1].astype(np.int64)).cuda()
    vals = rho[i, j].cpu().numpy()
    assert np.abs(vals - (s[:, 2] + 1j * s[:, 3])).max() <= 1e-9
    na, nb = api.observables(LARGE.params.Nc, LARGE.params.Nm, rho.t().contiguous().view(-1))
    assert abs(nb - ref["n_b"]) <= 1e-9 * abs(ref["n_b"]) + 1e-12
