"""om_ilu_apply_noalloc, the allocation-free preconditioner solve, against
om_ilu_apply (both called through the C ABI).

It serves callers that cannot allocate device memory (memory owned by
another allocator, or latency-critical code that must not enter the
allocator); its scratch is a static device array shared by all calls.  The
two entry points run the same sweep kernels, so their outputs must agree to
the tolerance used for repeated sweeps; two calls in a row check that the
contents a previous call leaves in the shared scratch do not leak into the
next result.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1411_4356_gb300 import _lib, api
from paper_1411_4356_gb300.workloads import SystemParams

pytestmark = pytest.mark.gpu

BASE = dict(omega_m=1.0, Delta=-1.0, kappa=0.5, g0=0.3, E=0.2, Q_m=1e3, n_th=0.5)


def call(name, M, flags, v, z):
    lib = _lib.load()
    st = getattr(lib, name)(M.handle, flags, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("Nc,Nm,d,fill", [(4, 10, 1e-4, 10.0), (6, 20, 1e-4, 20.0)])
def test_noalloc_matches_ilu_apply(Nc, Nm, d, fill):
    p = SystemParams(Nc, Nm, **BASE)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, d, fill, adjoint=True, fp64_sweeps=True)
    rng = np.random.default_rng(11)
    for flags in (0, 1, 2, 3):  # complex64 / complex128 sweeps, plain / conjugate transpose
        ref = torch.empty(Ar.N, dtype=torch.complex128, device="cuda")
        for call_no in range(2):
            v = torch.from_numpy(rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)).cuda()
            assert call("om_ilu_apply", M, flags | 4, v, ref) == 0  # bit 2: one-block sweeps, as noalloc
            z = torch.full_like(v, complex("nan"))
            assert call("om_ilu_apply_noalloc", M, flags, v, z) == 0, _lib.load().om_last_error()
            torch.cuda.synchronize()
            r, zz = ref.cpu().numpy(), z.cpu().numpy()
            assert np.all(np.isfinite(zz))
            np.testing.assert_allclose(zz, r, rtol=0, atol=1e-12 * np.abs(r).max())


def test_noalloc_after_a_larger_call():
    """A call on a 14,400-row factor, then one on a 1,600-row factor: the
    second must not see what the first left in the shared scratch beyond its
    own rows."""
    rng = np.random.default_rng(5)
    for (Nc, Nm, d, fill) in [(6, 20, 1e-4, 20.0), (4, 10, 1e-4, 10.0)]:
        p = SystemParams(Nc, Nm, **BASE)
        A = api.build_liouvillian(p)
        Ar, perm = api.permute(A)
        M = api.ilu_factor(Ar, d, fill, adjoint=True)
        for flags in (0, 2):
            v = torch.from_numpy(rng.standard_normal(Ar.N) + 1j * rng.standard_normal(Ar.N)).cuda()
            ref = torch.empty_like(v)
            assert call("om_ilu_apply", M, flags | 4, v, ref) == 0
            z = torch.full_like(v, complex("nan"))
            assert call("om_ilu_apply_noalloc", M, flags, v, z) == 0, _lib.load().om_last_error()
            torch.cuda.synchronize()
            r, zz = ref.cpu().numpy(), z.cpu().numpy()
            np.testing.assert_allclose(zz, r, rtol=0, atol=1e-12 * np.abs(r).max())


def test_noalloc_rejects_oversized_factor():
    p = SystemParams(10, 110, **BASE)  # 1,210,000 rows > 1,048,576
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    M = api.ilu_factor(Ar, 0.5, 1.0)
    v = torch.zeros(Ar.N, dtype=torch.complex128, device="cuda")
    z = torch.zeros_like(v)
    assert call("om_ilu_apply_noalloc", M, 0, v, z) == -1
    assert b"1048576" in _lib.load().om_last_error()
