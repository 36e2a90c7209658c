"""Adjoint gradients with the no-jump preconditioner on the 1,440,000-row
system (N_c = 12, N_m = 100, g0 = 1, n_th = 0.5): d<b^dag b>/dtheta and
d<a^dag a>/dtheta for theta = (Delta, E, g0, kappa) against central
differences of GPU forward solves (each perturbed system assembled and
factored afresh, solved to eta <= 1e-15), Richardson-extrapolated from steps
h and h/2 with h = 1e-4 (relative error O(h^4) ~ 1e-16 times the fourth
derivative, far below the tolerance).  The target is 1e-6 relative."""
import numpy as np
import pytest
import torch

from paper_1411_4356_gb300 import ADJOINT, api

pytestmark = pytest.mark.gpu

THETA = ("Delta", "E", "g0", "kappa")


def observable(p, rho, which):
    n = p.Nc * p.Nm
    h = torch.arange(n, device="cuda")
    q = (h // p.Nm) if which == "n_a" else (h % p.Nm)
    return float((torch.diagonal(rho).real * q).sum())


def solve(p, tol=1e-15, eig32=True):
    A = api.build_liouvillian(p, ADJOINT.trace_mode, ADJOINT.nth_floor)
    M = api.nojump_factor(p, nth_floor=ADJOINT.nth_floor, adjoint=True, eig32=eig32)
    rho, info = api.steady_state_solve_nojump(A, M, restart=50, tol=tol, max_iters=600, raise_on_noconv=False)
    assert info.eta <= 1e-14, info
    return A, M, rho


@pytest.mark.parametrize("which", ["n_b", "n_a"])
def test_adjoint_1440k_rows_against_central_differences(which):
    p = ADJOINT.params
    # the adjoint solve keeps a complex128 eigendecomposition (its preconditioner
    # is then accurate to ~1e-6, against ~3e-3 from a complex64 one) and asks a
    # relative residual of 1e-11: |mu| is large along the slow mechanical modes,
    # so the attainable residual is near 1e-12
    A, M, rho = solve(p, eig32=False)
    n = p.Nc * p.Nm
    h = torch.arange(n, device="cuda")
    q = ((h // p.Nm) if which == "n_a" else (h % p.Nm)).to(torch.complex128)
    g, ainfo = api.steady_state_adjoint_nojump(A, M, rho, torch.diag(q), restart=50, tol=1e-11, max_iters=600)

    def F(**kw):
        _, _, r = solve(p.with_(**kw))
        return observable(p, r, which)

    for t, name in enumerate(THETA):
        v = getattr(p, name)
        c = lambda hh: (F(**{name: v + hh}) - F(**{name: v - hh})) / (2 * hh)  # noqa: E731
        fd = (4 * c(5e-5) - c(1e-4)) / 3
        print(f"{which} d/d{name}: adjoint {g[t]:.12e} fd {fd:.12e} rel {abs(g[t] - fd) / abs(fd):.1e}")
        assert g[t] == pytest.approx(fd, rel=1e-6), (name, g[t], fd)
