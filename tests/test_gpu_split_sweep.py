"""The split triangular sweep (helper blocks sum the far slots of each tile,
the main block runs the dependency chain) against the oracle's ILUT solves
and against the one-block sweep.  Both sum the same complex64 products, in a
different order, so they agree to complex64 rounding amplified by the
factors."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle.reorder_factor import ilut
from paper_1411_4356_gb300 import MID, api
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


def gpu_csr(A):
    rp, ci, va = A.export()
    return sp.csr_matrix((va, ci, rp), shape=(A.N, A.N))


def split_launches(fn):
    api.profile(True)
    out = fn()
    torch.cuda.synchronize()
    _, n = api.profile_read(api.PROF_SPLIT)
    api.profile(False)
    return out, n


@pytest.mark.parametrize("Nc,Nm,d,fill", [(6, 20, 1e-4, 20.0), (6, 11, 1e-4, 20.0)])
def test_split_sweep_matches_oracle(Nc, Nm, d, fill):
    """14,400 rows (450 tiles) and 4,356 rows (136 tiles and a ragged tail of 4)."""
    p = SystemParams(Nc, Nm, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, d, fill, adjoint=True)
    F = ilut(gpu_csr(Ar), d, fill)
    rng = np.random.default_rng(Nc * 1000 + Nm)
    v = rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)
    vt = torch.from_numpy(v).cuda()
    for h in (False, True):
        ref = F.solve_h(v) if h else F.solve(v)
        z, n = split_launches(lambda: api.ilu_apply(M, vt, conj_transpose=h))
        z1 = api.ilu_apply(M, vt, conj_transpose=h, single_block=True)
        z, z1 = z.cpu().numpy(), z1.cpu().numpy()
        assert np.all(np.isfinite(z))
        scale = np.abs(ref).max()
        assert np.abs(z - ref).max() <= 1e-3 * scale
        assert np.abs(z - z1).max() <= 1e-3 * scale
        if Nm == 20:
            assert n == 2  # both sweeps ran split


def test_split_sweep_at_the_360k_structure():
    """N_c = 10, N_m = 20 with the 360,000-row system's parameters and
    ILUT(1e-5, 100): 1,250 tiles whose far slots outnumber the near ones.  The
    split and one-block sweeps agree, repeated applications are identical,
    and a solve through the split sweeps reaches its tolerance."""
    p = MID.params.with_(Nm=20)
    A = api.build_liouvillian(p, MID.trace_mode, MID.nth_floor)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, MID.droptol, MID.fill)
    rng = np.random.default_rng(20)
    vt = torch.from_numpy(rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)).cuda()
    z, n = split_launches(lambda: api.ilu_apply(M, vt))
    assert n == 2
    z2 = api.ilu_apply(M, vt)
    z1 = api.ilu_apply(M, vt, single_block=True)
    assert torch.isfinite(z).all()
    assert torch.equal(z, z2)  # fixed summation order: deterministic
    scale = float(z1.abs().max())
    assert float((z - z1).abs().max()) <= 1e-3 * scale
    (rho, info), n = split_launches(lambda: api.steady_state_solve(Ar, M, perm, restart=50, tol=1e-11))
    assert n >= 2 * info.iterations
    assert info.status == 0 and info.eta <= 1e-11
    assert abs(float(torch.trace(rho).real) - 1.0) < 1e-12
