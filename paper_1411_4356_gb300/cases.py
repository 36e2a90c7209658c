"""Named small cases for profiling single kernels (ncu captures).

    python -m paper_1411_4356_gb300.cases sweep_10x20

builds the 40,000-row Liouvillian (N_c = 10, N_m = 20, the 360,000-row
system's parameters), permutes it, factors it (d = 1e-5, p = 100) and runs
the complex64 preconditioner solve three times; `spmv_10x60` runs the SpMV
three times instead.  Inputs are larger than L2 (the factors are ~0.4 GB).
`batched_16` solves the first 16 draws of the 512-system sweep with the
lock-step batched engine.  `nojump_20x100` factors K of the 4,000,000-row
system (N_c = 20, N_m = 100, the 16M-row system's parameters) and applies the
no-jump preconditioner three times with the TF32 tensor-core products (each
expanded operand 64 MB, each data matrix 32 MB: larger than L2 together).
`solve_20x100` / `solve_mixed_20x100` run the whole no-jump steady-state solve
of that system in FP64 / mixed precision (Krylov basis 3.3 GB / 1.6 GB).
"""
from __future__ import annotations

import sys

import torch

from . import api
from .workloads import MID


def _system(Nc, Nm):
    p = MID.params.with_(Nc=Nc, Nm=Nm)
    A = api.build_liouvillian(p)
    Ar, perm = api.permute(A)
    return p, Ar, perm


def sweep(Nc=10, Nm=20):
    p, Ar, perm = _system(Nc, Nm)
    M = api.ilu_factor(Ar, MID.droptol, MID.fill)
    x = torch.randn(Ar.N, dtype=torch.complex128, device="cuda")
    for _ in range(3):
        api.ilu_apply(M, x)
    torch.cuda.synchronize()
    print(f"sweep case: rows {Ar.N}, nnz(L) {M.nnz_l}, nnz(U) {M.nnz_u}, levels {M.levels_l}/{M.levels_u}")


def spmv(Nc=10, Nm=60):
    p, Ar, perm = _system(Nc, Nm)
    x = torch.randn(Ar.N, dtype=torch.complex128, device="cuda")
    for _ in range(3):
        api.spmv(Ar, x)
    torch.cuda.synchronize()
    print(f"spmv case: rows {Ar.N}, nnz {Ar.nnz}")


def batched(count=16):
    from .workloads import BATCH, batched_draws

    systems = []
    for p in batched_draws(count):
        A = api.build_liouvillian(p, BATCH.trace_mode, BATCH.nth_floor)
        Ar, perm = api.permute(A)
        M = api.ilu_factor(Ar, BATCH.droptol, BATCH.fill)
        if not (api.ilu_condest(M) < 1e12):
            M = api.ilu_factor(Ar, BATCH.droptol, BATCH.refill)
        systems.append((Ar, M, perm))
    _, infos = api.steady_state_solve_batched(systems, restart=BATCH.restart, tol=BATCH.tol)
    torch.cuda.synchronize()
    print(f"batched case: {count} systems, iterations {[i.iterations for i in infos]}")


def nojump(Nc=20, Nm=100):
    from .workloads import LARGE

    p = LARGE.params.with_(Nc=Nc, Nm=Nm)
    M = api.nojump_factor(p, nth_floor=LARGE.nth_floor, eig32=True)
    x = torch.randn(p.N, dtype=torch.complex128, device="cuda")
    for _ in range(3):
        api.nojump_apply(M, x)
    torch.cuda.synchronize()
    print(f"nojump case: n {p.n}, rows {p.N}, tensor cores {M.tensor_cores}")


def solve(Nc=20, Nm=100, precision=0):
    from .workloads import LARGE

    p = LARGE.params.with_(Nc=Nc, Nm=Nm)
    A = api.build_liouvillian(p, LARGE.trace_mode, LARGE.nth_floor)
    M = api.nojump_factor(p, nth_floor=LARGE.nth_floor, eig32=True)
    rho, info = api.steady_state_solve_nojump(A, M, restart=50, tol=1e-12, precision=precision)
    torch.cuda.synchronize()
    print(f"solve case: rows {p.N}, precision {precision}, iterations {info.iterations}, eta {info.eta:.2e}")


CASES = {"sweep_10x20": lambda: sweep(10, 20), "spmv_10x60": lambda: spmv(10, 60), "batched_16": batched,
         "nojump_20x100": lambda: nojump(20, 100), "solve_20x100": lambda: solve(20, 100, 0),
         "solve_mixed_20x100": lambda: solve(20, 100, 1)}

if __name__ == "__main__":
    CASES[sys.argv[1]]()
