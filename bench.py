"""Benchmark: steady-state solves/s of the driven, damped optomechanical
system, mixed precision against FP64, at eta <= tol (default 1e-12, so that
rho also matches the oracle to 1e-9; the metric's residual is 1e-10).

Default workload: N_c = 20, N_m = 200 (Liouvillian 16,000,000 rows, 183M
nonzeros), g0 = 1.5, n_th = 0 floored to 1e-15 (Sec. IV), mixed precision.
One step is one pass of the whole path on the GPU through the C ABI:
assemble L~ (Eq. 1-5) -> K = -i H - (1/2) sum gamma O^dag O and its
eigendecomposition (the no-jump preconditioner) -> GMRES (Sec. IV) with
complex64 inner iterations inside FP64 refinement -> trace normalisation ->
<a^dag a>, <b^dag b>.  The same line reports the FP64 form of the same step,
the 360,000-row system (N_c = 10, N_m = 60) with the no-jump preconditioner and
with the paper's RCM + ILUT preconditioner, parity against the stored oracle
references, the roofline of the dominant kernel and the oracle on the host
cores.  Inputs are the system parameters; the working set (Krylov basis of
several GB) is far larger than L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl omss|reference]
                    [--workload large|mid|mid_ilu|batched|sweep]

For N > 1 launch with torch.distributed.run: every rank solves its own
system (independent replicas, weak scaling).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the batched sweep runs one stream per concurrent solve; let CUDA map them to
# 32 hardware queues instead of 8 (must be set before CUDA initialises)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "steady-state solves/s & Krylov HBM GB/s, mixed vs FP64 at residual 1e-10"
RESTART = 50  # GMRES restart of the no-jump solves


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["omss", "reference"], default="omss")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline workload only (no FP64 / 360k sub-lines)")
    ap.add_argument("--tol", type=float, default=1e-12, help="eta target of the benched solves")
    ap.add_argument("--workload", choices=["large", "mid", "mid_ilu", "batched", "sweep"], default="large",
                    help="large: 16M rows, mixed precision (default); mid: 360,000 rows, FP64, no-jump "
                         "preconditioner; mid_ilu: 360,000 rows with the paper's RCM + ILUT; batched: the "
                         "parameter sweep (N_c = 6, N_m in {20, 30, 40, 60}), solve phase timed")
    ap.add_argument("--systems", type=int, default=64, help="systems of the sweep for --workload batched")
    ap.add_argument("--concurrency", type=int, default=0,
                    help="--workload batched: 0 = lock-step engine, k > 0 = k concurrent single solves")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                pass
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def source_hash(*paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sweep_traffic_per_entry(kernel_hash: str, name: str = "sweep_traffic.json"):
    """DRAM bytes per stored factor entry of one sweep launch, from a
    committed ncu summary of the 40,000-row case, or None if the kernel
    source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("sweep_source_hash") != kernel_hash:
        return None
    return d.get("dram_bytes_per_factor_entry")


def max_over_ranks(values, world: int, dist=None):
    """Element-wise maximum of per-rank timings (every rank gets the result)."""
    if world <= 1:
        return list(values)
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


# ----------------------------------------------------------------- GPU arm
def golden(name):
    path = os.path.join(ROOT, "tests", "golden", name)
    return json.load(open(path)) if os.path.exists(path) else None


def parity_vs(ref, rho_dev, n):
    """max |rho_ij - rho_oracle| over the stored diagonal and sampled entries."""
    if ref is None:
        return None
    import torch

    r = rho_dev.view(n, n).t()  # r[i, j] = rho_ij
    diag = torch.diagonal(r).cpu().numpy()
    d = np.abs(diag - (np.array(ref["diag_re"]) + 1j * np.array(ref["diag_im"]))).max()
    s = np.array(ref["samples"])
    i, j = torch.from_numpy(s[:, 0].astype(np.int64)), torch.from_numpy(s[:, 1].astype(np.int64))
    vals = r[i.cuda(), j.cuda()].cpu().numpy()
    e = np.abs(vals - (s[:, 2] + 1j * s[:, 3])).max()
    return {"max_abs_err": float(max(d, e)), "entries_compared": int(len(diag) + len(s)),
            "oracle_eta": ref.get("eta", ref.get("solver", {}).get("eta"))}


def invariants(rho_dev, p):
    """Trace, Hermiticity and the exact truncated identity kappa <a^dag a> = -2 E Im<a>."""
    import torch

    n = p.Nc * p.Nm
    r = rho_dev.view(n, n).t()
    tr = complex(torch.diagonal(r).sum().item())
    herm = float((r - r.conj().t()).abs().max().item())
    c = torch.arange(n, device=r.device) // p.Nm
    na = float((torch.diagonal(r).real * c).sum().item())
    # <a> = sum_h sqrt(c+1) rho_{(c+1,m),(c,m)}: a |c+1, m> = sqrt(c+1) |c, m>
    h = torch.arange(n - p.Nm, device=r.device)
    a_exp = complex((torch.sqrt((h // p.Nm + 1).double()) * r[h + p.Nm, h]).sum().item())
    return {"trace_minus_1": abs(tr - 1), "max_hermiticity": herm,
            "kappa_na_plus_2E_im_a": abs(p.kappa * na + 2 * p.E * a_exp.imag)}


class NojumpStep:
    """One pass of the no-jump path: assemble, factor K, solve, observables."""

    def __init__(self, w, precision, tol, rho_dev, restart=RESTART, eig32=True):
        self.w, self.precision, self.tol, self.rho_dev = w, precision, tol, rho_dev
        self.restart, self.eig32 = restart, eig32

    def __call__(self):
        from paper_1411_4356_gb300 import api

        w, p = self.w, self.w.params
        h0 = time.perf_counter()
        A = api.build_liouvillian(p, w.trace_mode, w.nth_floor)
        h1 = time.perf_counter()
        M = api.nojump_factor(p, nth_floor=w.nth_floor, eig32=self.eig32)
        h2 = time.perf_counter()
        _, info = api.steady_state_solve_nojump(A, M, restart=self.restart, tol=self.tol, precision=self.precision,
                                                rho_out=self.rho_dev, max_iters=12000)
        obs = api.observables(p.Nc, p.Nm, self.rho_dev)
        P, mean, second, fano = api.phonon_distribution(p.Nc, p.Nm, self.rho_dev)
        st = dict(N=A.N, nnz=A.nnz, iterations=info.iterations, cycles=info.cycles, eta=info.eta,
                  solve_s=info.seconds, build_s=h1 - h0, factor_s=h2 - h1, factor_phases=M.timings,
                  tensor_cores=M.tensor_cores, min_abs_d=M.min_abs_d, obs=obs, P=P, fano=fano)
        M.free()
        A.free()
        return st


def ilu_step(w, rho_dev, tol):
    """The paper's path on the 360,000-row system: RCM, ILUT(1e-5, 100), GMRES(50)."""
    from paper_1411_4356_gb300 import api

    p = w.params
    h0 = time.perf_counter()
    A = api.build_liouvillian(p, w.trace_mode, w.nth_floor)
    Ar, perm = api.permute(A)
    A.free()
    M = api.ilu_factor(Ar, w.droptol, w.fill)
    _, info = api.steady_state_solve(Ar, M, perm, restart=w.restart, tol=tol, rho_out=rho_dev)
    st = dict(iterations=info.iterations, eta=info.eta, solve_s=info.seconds, ilu_s=M.timings, fill=M.fill,
              levels=(M.levels_l, M.levels_u), nnz_l=M.nnz_l, nnz_u=M.nnz_u, N=Ar.N,
              wall_s=time.perf_counter() - h0)
    M.free()
    Ar.free()
    return st


def timed(fn, stream, reps=1):
    """CUDA-event time (s) of reps calls of fn on `stream`, and the last result."""
    import torch

    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps, out


def measured_peak_tf32():
    """TF32 dense peak: the measured bf16 peaks (burst, sustained) x the nominal
    tf32 / bf16 ratio 1.1 / 2.25 PFLOP/s."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    ratio = 1.1 / 2.25
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["bf16_tflops"]) * ratio, float(d["bf16_tflops_sustained"]) * ratio, "measured"
    return 1900.0 * ratio, 1700.0 * ratio, "fallback"


def krylov_bytes(its, cycles, restart, N, vec_bytes):
    """Algorithmic bytes of the CGS2 passes over a solve: per step j (1-based
    basis of j vectors) two passes, each a multi-dot (j vectors + w read) and
    an update (j vectors + w read, w written).  The iterations are taken as
    evenly split over the cycles (GMRES restarts or refinement steps), each
    cycle starting a new basis."""
    total = 0
    cycles = max(1, cycles)
    for c in range(cycles):
        its_c = its // cycles + (1 if c < its % cycles else 0)
        j = 0
        for _ in range(its_c):
            j = j % restart + 1
            total += 2 * (2 * j + 3) * vec_bytes * N
    return total


def run_omss(args):
    import torch
    import torch.distributed as dist

    from paper_1411_4356_gb300 import LARGE, MID, api

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    if args.workload == "mid_ilu":
        return run_mid_ilu(args, world, rank, dist)
    w = LARGE if args.workload == "large" else MID
    precision = 1 if args.workload == "large" else 0
    p = w.params
    n = p.Nc * p.Nm
    rho_dev = torch.empty(n * n, dtype=torch.complex128, device="cuda")
    rho_host = torch.empty(n * n, dtype=torch.complex128, pin_memory=True)
    step = NojumpStep(w, precision, args.tol, rho_dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- timed region: K steps between CUDA events (inputs resident: the
    # parameters); e2e adds the read-back of rho to pinned host memory each step
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = api.kernel_launches()
    api.profile(True)
    stats = []
    device_s = 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dt, st = timed(step, stream)
        device_s += dt
        rho_host.copy_(rho_dev, non_blocking=True)
        torch.cuda.synchronize()
        stats.append(st)
    e2e_s = time.perf_counter() - t0
    barrier()
    launches = api.kernel_launches() - launches0
    prof = {name: api.profile_read(c) for name, c in
            (("nojump", api.PROF_NOJUMP), ("stencil", api.PROF_STENCIL), ("krylov", api.PROF_KRYLOV))}
    api.profile(False)
    clk = clocks.stop()
    elapsed, e2e_s = max_over_ranks([device_s, e2e_s], world, dist)
    s0 = stats[-1]
    parity = parity_vs(golden("large_20x200_reference.json" if w is LARGE else "mid_10x60_reference.json"),
                       rho_dev, n)
    inv = invariants(rho_dev, p)
    rho_mixed = rho_dev.clone()

    extras = {}
    if not args.no_extras:
        # the same step in FP64 throughout the Krylov iteration (the comparison the metric asks for)
        other = 0 if precision == 1 else 1
        dt, st = timed(NojumpStep(w, other, args.tol, rho_dev), stream)
        extras["fp64" if other == 0 else "mixed"] = {
            "value": world / dt, "unit": "solves/s", "ms_per_step": dt * 1e3, "iterations": st["iterations"],
            "cycles": st["cycles"], "eta": st["eta"], "solve_s": st["solve_s"],
            "max_abs_diff_vs_headline_rho": float((rho_dev - rho_mixed).abs().max().item()),
            "parity": parity_vs(golden("large_20x200_reference.json" if w is LARGE else "mid_10x60_reference.json"),
                                rho_dev, n)}
        if w is LARGE:
            # the 360,000-row system: no-jump FP64 (3 steps) and the paper's RCM + ILUT path (1 step)
            nm = MID.params.Nc * MID.params.Nm
            rho_mid = torch.empty(nm * nm, dtype=torch.complex128, device="cuda")
            mstep = NojumpStep(MID, 0, args.tol, rho_mid)
            mstep()
            dt, st = timed(mstep, stream, reps=3)
            extras["mid_10x60"] = {
                "value": world / dt, "unit": "solves/s", "ms_per_step": dt * 1e3, "iterations": st["iterations"],
                "eta": st["eta"], "solve_s": st["solve_s"], "factor_s": st["factor_s"],
                "precision": "FP64 flexible GMRES, TF32 no-jump products",
                "parity": parity_vs(golden("mid_10x60_reference.json"), rho_mid, nm)}
            # the paper's application (Sec. V, Fig. 5): the c-CPT at 640,000 rows
            from paper_1411_4356_gb300 import CCPT

            nc = CCPT.params.Nc * CCPT.params.Nm
            rho_cc = torch.empty(nc * nc, dtype=torch.complex128, device="cuda")
            cstep = NojumpStep(CCPT, CCPT.precision, CCPT.tol, rho_cc, restart=CCPT.restart, eig32=False)
            cstep()
            dt, st = timed(cstep, stream, reps=2)
            ref = golden("ccpt_5x160_reference.json")
            extras["ccpt_5x160"] = {
                "value": world / dt, "unit": "solves/s", "ms_per_step": dt * 1e3, "iterations": st["iterations"],
                "eta": st["eta"], "tol": CCPT.tol, "solve_s": st["solve_s"], "factor_s": st["factor_s"],
                "precision": "complex64 GMRES(120) in FP64 refinement, TF32 no-jump products",
                "n_b": st["obs"][1], "fano": st["fano"],
                "parity": None if ref is None else dict(
                    parity_vs(ref, rho_cc, nc),
                    max_abs_err_P=float(np.abs(st["P"] - np.array(ref["P"])).max()),
                    oracle_fano=ref["fano"], oracle_eta=ref["eta"])}
            del rho_cc
            # the adjoint configuration (1.44M rows): forward solve, then the
            # adjoint solve for d<b^dag b>/d(Delta, E, g0, kappa); a central
            # difference in E as a check
            from paper_1411_4356_gb300 import ADJOINT

            def adjoint_step():
                q = ADJOINT.params
                Aa = api.build_liouvillian(q, ADJOINT.trace_mode, ADJOINT.nth_floor)
                Ma = api.nojump_factor(q, nth_floor=ADJOINT.nth_floor, adjoint=True)
                ra, ia = api.steady_state_solve_nojump(Aa, Ma, restart=RESTART, tol=1e-13, max_iters=600)
                hh = torch.arange(q.n, device="cuda")
                G = torch.diag((hh % q.Nm).to(torch.complex128))
                g, ga = api.steady_state_adjoint_nojump(Aa, Ma, ra, G, restart=RESTART, tol=1e-11, max_iters=600)
                out = dict(forward_iterations=ia.iterations, adjoint_iterations=ga.iterations, eta=ia.eta,
                           gradient_n_b=dict(zip(("Delta", "E", "g0", "kappa"), [float(x) for x in g])))
                Ma.free()
                Aa.free()
                return out

            adjoint_step()
            dt, st = timed(adjoint_step, stream)

            def n_b_at(**kw):
                q = ADJOINT.params.with_(**kw)
                Aq = api.build_liouvillian(q, ADJOINT.trace_mode, ADJOINT.nth_floor)
                Mq = api.nojump_factor(q, nth_floor=ADJOINT.nth_floor)
                rq, _ = api.steady_state_solve_nojump(Aq, Mq, restart=RESTART, tol=1e-14, max_iters=600)
                return api.observables(q.Nc, q.Nm, rq)[1]

            hE = 1e-4
            fdE = (n_b_at(E=ADJOINT.params.E + hE) - n_b_at(E=ADJOINT.params.E - hE)) / (2 * hE)
            extras["adjoint_12x100"] = {
                "value": world / dt, "unit": "gradients/s (4 parameters, one observable)", "ms_per_step": dt * 1e3,
                **st, "fd_check": {"parameter": "E", "central_difference": fdE, "step": hE,
                                   "rel_diff": abs(st["gradient_n_b"]["E"] - fdE) / abs(fdE)}}
            # the 512-system parameter sweep, each system through the whole no-jump path
            from paper_1411_4356_gb300.workloads import batched_draws

            sp_params = sorted(batched_draws(512), key=lambda q: -q.Nm)
            sweep_pass(sp_params[:32], 16)  # warm-up
            dt, infos, rhos = sweep_pass(sp_params, 16)
            extras["sweep_512"] = {"value": len(sp_params) / dt, "unit": "solves/s", "ms_per_step": dt * 1e3,
                                   "systems": len(sp_params), "concurrency": 16,
                                   "precision": "complex64 GMRES(50) in FP64 refinement, TF32 no-jump products",
                                   **sweep_summary(sp_params, infos, rhos)}
            del rhos
            api.profile(True)
            dt, st = timed(lambda: ilu_step(MID, rho_mid, args.tol), stream)
            sp_ms, sp_n = api.profile_read(api.PROF_SPLIT)
            api.profile(False)
            extras["mid_10x60_paper_ilu"] = {
                "value": world / dt, "unit": "solves/s", "ms_per_step": dt * 1e3, "iterations": st["iterations"],
                "eta": st["eta"], "solve_s": st["solve_s"], "ilut_host_s": st["ilu_s"]["ilut"], "fill": st["fill"],
                "levels": st["levels"], "split_sweep_avg_ms": sp_ms / max(sp_n, 1),
                "preconditioner": "RCM (Sec. III) + ILUT(1e-5, 100) (Sec. II), complex64 split sweeps",
                "parity": parity_vs(golden("mid_10x60_reference.json"), rho_mid, nm)}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    N = s0["N"]
    its = s0["iterations"]
    solve_s = statistics.mean(st["solve_s"] for st in stats)
    vec_bytes = 8 if precision == 1 else 16
    # per-kernel device time over the timed steps
    nj_ms, nj_n = prof["nojump"]
    st_ms, st_n = prof["stencil"]
    kr_ms, kr_n = prof["krylov"]
    flops_apply = 4 * 8.0 * n ** 3  # four complex n x n products, 8 n^3 real flops each
    tc_achieved = flops_apply * nj_n / (nj_ms / 1e3) / 1e12 if nj_ms > 0 else 0.0
    tf32_burst, tf32_sust, peak_kind = measured_peak_tf32()
    cgs_bytes = krylov_bytes(its, s0["cycles"], RESTART, N, vec_bytes) * args.steps
    sten_bytes = 2 * vec_bytes * N * st_n  # read x, write y per application
    hbm, hbm_kind = measured_peaks()
    shares = {"nojump_products": nj_ms, "gram_schmidt": kr_ms, "stencil_operator": st_ms}
    dominant = max(shares, key=shares.get)
    tc_roof = {"bound": "tensor", "kernel": "tc_product (TF32 tcgen05 complex products of the no-jump preconditioner)",
               "achieved": tc_achieved, "peak": tf32_sust, "unit": "TFLOP/s", "frac": tc_achieved / tf32_sust,
               "peak_kind": f"{peak_kind} bf16 sustained x nominal tf32/bf16 (1.1/2.25)",
               "traffic": tc_traffic_per_launch(), "avg_launch_ms": nj_ms / max(nj_n, 1) / 4, "launches": 4 * nj_n,
               "flops_per_launch": flops_apply / 4}
    cgs_gbs = cgs_bytes / (kr_ms / 1e3) / 1e9 if kr_ms > 0 else 0.0
    cgs_roof = {"bound": "hbm", "kernel": "multidot_rows + multi_axpy_rows (CGS2 Gram-Schmidt of the GMRES step)",
                "achieved": cgs_gbs, "peak": hbm, "unit": "GB/s", "frac": cgs_gbs / hbm,
                "peak_kind": f"{hbm_kind} copy bandwidth", "traffic": None,
                "avg_launch_ms": kr_ms / max(kr_n, 1) / 4, "launches": 4 * kr_n,
                "bytes_per_launch": cgs_bytes / max(4 * kr_n, 1)}
    sten_gbs = sten_bytes / (st_ms / 1e3) / 1e9 if st_ms > 0 else 0.0
    sten_roof = {"bound": "hbm", "kernel": "stencil_apply (L~ x from the stencil of Eq. 3)", "achieved": sten_gbs,
                 "peak": hbm, "unit": "GB/s", "frac": sten_gbs / hbm, "avg_launch_ms": st_ms / max(st_n, 1),
                 "launches": st_n}
    parts = {"nojump_products": tc_roof, "gram_schmidt": cgs_roof, "stencil_operator": sten_roof}
    roofline = dict(parts[dominant])
    roofline["device_ms_by_part"] = shares
    roofline["dominant_part"] = dominant
    roofline["other_parts"] = {k: v for k, v in parts.items() if k != dominant}
    line = {
        "metric": METRIC,
        "value": args.steps * world / elapsed,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("c64 Krylov + TF32 products inside c128 refinement" if precision == 1
                  else "c128 Krylov + TF32 preconditioner products"),
        "data": "synthetic",
        "config": {"workload": w.name, "Nc": p.Nc, "Nm": p.Nm, "rows": N, "nnz": s0["nnz"], "g0": p.g0,
                   "n_th": p.n_th, "nth_floor": w.nth_floor, "precision": "mixed" if precision == 1 else "fp64",
                   "preconditioner": "no-jump: exact inverse of K rho + rho K^dag (eigendecomposition, complex64)",
                   "restart": RESTART, "tol": args.tol, "trace_mode": w.trace_mode,
                   "parallelism": f"replicas x{world}",
                   "l2": "working set (Krylov basis, GB) larger than L2; no flush needed"},
        "roofline": roofline,
        "e2e": {"value": args.steps * world / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 72 + 16,
                "d2h_bytes_per_step": 16 * n * n},
        "gpu_launches": int(launches),
        "clocks": clk,
        "krylov_iterations_per_s": its / solve_s,
        "krylov_gbs": (cgs_bytes + sten_bytes) / ((kr_ms + st_ms) / 1e3) / 1e9 if kr_ms + st_ms > 0 else None,
        "iterations": its,
        "cycles": s0["cycles"],
        "eta": s0["eta"],
        "parity": parity,
        "invariants": inv,
        "phase_s": {"build": statistics.mean(st["build_s"] for st in stats),
                    "factor": statistics.mean(st["factor_s"] for st in stats), "solve": solve_s},
        "observables": {"n_a": s0["obs"][0], "n_b": s0["obs"][1]},
        **extras,
    }
    if world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(w, line["iterations"])
        line["cpu_baseline"] = {"value": cb["value"], "unit": "solves/s", "cores": cb["cores"], "kind": "oracle",
                                "sample": cb["sample"]}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def tc_traffic_per_launch():
    """DRAM bytes per launch of the tensor-core product at the 16M-row size,
    from a committed ncu summary, or None if nojump_tc.cu changed since."""
    path = os.path.join(ROOT, "profiles", "tc_product_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("source_hash") != source_hash(os.path.join(ROOT, "paper_1411_4356_gb300", "csrc", "nojump_tc.cu")):
        return None
    return d.get("dram_bytes_per_launch_large")


def run_mid_ilu(args, world, rank, dist):
    """The paper's RCM + ILUT path on the 360,000-row system as the benched step."""
    import torch

    from paper_1411_4356_gb300 import MID, api

    n = MID.params.Nc * MID.params.Nm
    rho_dev = torch.empty(n * n, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ilu_step(MID, rho_dev, args.tol)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    launches0 = api.kernel_launches()
    api.profile(True)
    elapsed, stats = 0.0, []
    for _ in range(args.steps):
        dt, st = timed(lambda: ilu_step(MID, rho_dev, args.tol), stream)
        elapsed += dt
        stats.append(st)
    split_ms, split_n = api.profile_read(api.PROF_SPLIT)
    api.profile(False)
    launches = api.kernel_launches() - launches0
    clk = clocks.stop()
    (elapsed,) = max_over_ranks([elapsed], world, dist)
    if rank != 0:
        return
    s0 = stats[-1]
    N = s0["N"]
    bytes_l = 12 * s0["nnz_l"] + 8 * (N + 1) + 16 * N
    bytes_u = 12 * (s0["nnz_u"] - N) + 8 * (N + 1) + 24 * N
    achieved = (bytes_l + bytes_u) / 2.0 * split_n / (split_ms / 1e3) / 1e9 if split_ms > 0 else 0.0
    peak, peak_kind = measured_peaks()
    line = {"metric": METRIC, "value": args.steps * world / elapsed, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128 Krylov + c64 ILU sweeps", "data": "synthetic",
            "config": {"workload": MID.name + "_paper_ilu", "droptol": MID.droptol, "fill_cap": MID.fill,
                       "restart": MID.restart, "tol": args.tol},
            "roofline": {"bound": "hbm", "kernel": "split_sweep", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} copy bandwidth",
                         "traffic": None, "avg_launch_ms": split_ms / max(split_n, 1), "launches": split_n},
            "gpu_launches": int(launches), "clocks": clk, "iterations": s0["iterations"], "eta": s0["eta"],
            "parity": parity_vs(golden("mid_10x60_reference.json"), rho_dev, n),
            "phase_s": {"ilut_host": s0["ilu_s"]["ilut"], "solve": s0["solve_s"]}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- oracle leg
def oracle_sample(w, gpu_iterations: int, samples: int = 1):
    """The FP64 oracle on the host cores, on a bounded sample of the same
    workload: the Schur form of K (the oracle's set-up of the no-jump
    preconditioner, timed in full) and `samples` applications of its
    Bartels-Stewart inverse (each the bulk of one oracle GMRES iteration),
    converted to solves/s with the oracle's own iteration count from its stored
    reference run (the GPU's count when no reference is stored).  Assembly,
    SpMV and Gram-Schmidt are not counted, so the figure is an upper bound on
    the oracle's solves/s."""
    from oracle.liouvillian import Params
    from oracle.nojump import NoJumpInverse

    p = w.params
    op = Params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th)
    ref = golden("large_20x200_reference.json" if w.name.startswith("large") else "mid_10x60_nojump_reference.json")
    its = int(ref["iterations"]) if ref and "iterations" in ref else gpu_iterations
    t0 = time.perf_counter()
    S = NoJumpInverse(op, w.nth_floor)
    t_schur = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    N = op.Nc * op.Nm * op.Nc * op.Nm
    y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    t_apply = []
    for _ in range(samples):
        t0 = time.perf_counter()
        S(y)
        t_apply.append(time.perf_counter() - t0)
    ta = statistics.mean(t_apply)
    total = t_schur + its * ta
    cores = os.cpu_count() or 1
    return {"value": 1.0 / total, "cores": cores, "seconds_per_solve": total, "t_schur": t_schur, "t_apply": ta,
            "iterations": its,
            "sample": (f"oracle no-jump preconditioner on the host cores ({cores} threads available to BLAS): "
                       f"Schur form of K (n = {op.Nc * op.Nm}) {t_schur:.1f} s and one FP64 Bartels-Stewart "
                       f"application {ta:.1f} s (mean of {samples}), x {its} iterations of the oracle's reference "
                       f"run; assembly, SpMV and Gram-Schmidt not counted (an upper bound on the oracle's rate)")}


def run_batched(args):
    """The parameter sweep: the first `systems` draws of the 512-system sweep,
    set up (assembly, RCM, ILUT) outside the timed region, then solved
    together with om_steady_state_solve_batched; K timed repetitions."""
    import torch

    from paper_1411_4356_gb300 import api
    from paper_1411_4356_gb300.workloads import BATCH, batched_draws

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    params = sorted(batched_draws(512)[: args.systems], key=lambda p: -p.Nm)
    t0 = time.perf_counter()
    systems = []
    refactored = 0
    for p in params:
        A = api.build_liouvillian(p, BATCH.trace_mode, BATCH.nth_floor)
        Ar, perm = api.permute(A)
        A.free()
        M = api.ilu_factor(Ar, BATCH.droptol, BATCH.fill)
        # Sec. IV's estimate ||(LU)^{-1} e||_inf flags an unstable factor
        # before any solve; those draws are refactored with the larger cap
        est = api.ilu_condest(M)
        if not (est < 1e12):
            M.free()
            M = api.ilu_factor(Ar, BATCH.droptol, BATCH.refill)
            refactored += 1
        systems.append((Ar, M, perm))
    setup_s = time.perf_counter() - t0
    def solve():
        return api.steady_state_solve_batched(systems, restart=BATCH.restart, tol=BATCH.tol,
                                              concurrency=args.concurrency)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = api.kernel_launches()
    api.profile(True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, infos = solve()
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    sweep_ms, sweep_n = api.profile_read(api.PROF_SWEEP)
    split_ms, split_n = api.profile_read(api.PROF_SPLIT)
    api.profile(False)
    launches = api.kernel_launches() - launches0
    clk = clocks.stop()
    # algorithmic bytes of the preconditioner applications: every application
    # streams the system's complex64 factors once (12 B per entry with its
    # column) plus the vector conversions; one per Krylov iteration
    swept = 0.0
    for (Ar, M, perm), info in zip(systems, infos):
        per_apply = 12 * (M.nnz_l + M.nnz_u - Ar.N) + 2 * (8 * (Ar.N + 1) + 16 * Ar.N)
        swept += per_apply * info.iterations
    swept *= args.steps
    engine = "lock-step" if args.concurrency <= 0 else f"{args.concurrency} concurrent streams"
    kernel = ("b_precond: one launch per Krylov step, one block per system; split_sweep for the last "
              "systems" if args.concurrency <= 0 else "tile_sweep, concurrent over the batch")
    # lock-step: the preconditioner launches (and the split sweeps of the last
    # systems, continued one by one) are timed themselves; streams: only the
    # wall clock of the batch bounds them
    sweep_s = (sweep_ms + split_ms) / 1e3 if args.concurrency <= 0 and sweep_ms > 0 else elapsed
    peak, peak_kind = measured_peaks()
    bad = [i.status for i in infos if i.status != 0]
    line = {"metric": METRIC, "value": len(systems) * args.steps / elapsed, "unit": "solves/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": BATCH.name, "systems": len(systems), "Nc": 6,
                       "Nm": sorted({p.Nm for p in params}), "rows_total": sum(A.N for A, _, _ in systems),
                       "droptol": BATCH.droptol, "fill_cap": BATCH.fill, "restart": BATCH.restart, "tol": BATCH.tol,
                       "timed": "batched solve phase (setup outside)", "setup_s": setup_s, "engine": engine,
                       "refactored_unstable": refactored, "refill_cap": BATCH.refill},
            "roofline": {"bound": "hbm", "kernel": kernel,
                         "achieved": swept / sweep_s / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": swept / sweep_s / 1e9 / peak, "peak_kind": f"{peak_kind} copy bandwidth",
                         "traffic": None, "sweep_launches": sweep_n,
                         "sweep_device_ms_sum": sweep_ms, "tail_split_sweeps": split_n,
                         "tail_split_ms_sum": split_ms},
            "gpu_launches": int(launches), "clocks": clk,
            "iterations": [i.iterations for i in infos], "failed": bad}
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The oracle on the host cores, on the same workload: one warm-up sample,
    then `steps` bounded samples (oracle_sample); each step is one sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1411_4356_gb300 import LARGE, MID

    w = LARGE if args.workload in ("large",) else MID
    steps = max(1, min(args.steps, 2))  # each sample takes about a minute at 16M rows
    t0 = time.perf_counter()
    vals = [oracle_sample(w, 50) for _ in range(steps)]
    wall = time.perf_counter() - t0
    value = statistics.mean(v["value"] for v in vals)
    cores = vals[-1]["cores"]
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "impl": "reference",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": steps, "warmup": 0,
            "ms_per_step": wall / steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": w.name, "Nc": w.params.Nc, "Nm": w.params.Nm,
                       "note": "one step = one bounded oracle sample (Schur form of K + one Bartels-Stewart "
                               "application); value converts it to solves/s with the oracle's iteration count"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sweep_pass(params, concurrency):
    """The 512-system parameter sweep through the whole no-jump path (assembly,
    K and its complex64 eigendecomposition, mixed GMRES to eta 1e-12) on
    concurrent streams: (seconds of the pass on the device clock, infos, rhos)."""
    import torch

    from paper_1411_4356_gb300 import api

    stream = torch.cuda.current_stream()
    dt, (rhos, infos) = timed(lambda: api.steady_state_sweep_nojump(params, restart=RESTART, tol=1e-12, precision=1,
                                                                    concurrency=concurrency, eig32=True), stream)
    return dt, infos, rhos


def sweep_summary(params, infos, rhos):
    """Statuses, iterations and the invariants of every system of a sweep."""
    import torch

    bad = [i for i, inf in enumerate(infos) if inf.status != 0]
    tr = max(abs(complex(torch.diagonal(r).sum().item()) - 1) for r in rhos)
    herm = max(float((r - r.conj().t()).abs().max().item()) for r in rhos)
    its = [inf.iterations for inf in infos]
    return {"failed": bad, "iterations_mean": float(np.mean(its)), "iterations_max": int(max(its)),
            "eta_max": float(max(inf.eta for inf in infos)), "max_trace_minus_1": tr, "max_hermiticity": herm,
            "rows_total": int(sum(p.N for p in params))}


def run_sweep(args):
    """--workload sweep: the first `systems` draws of the 512-system sweep
    (N_c = 6, Delta ~ U[-3, 1], N_m in {20, 30, 40, 60}), each through the whole
    no-jump path per step; K timed passes."""
    import torch

    from paper_1411_4356_gb300 import api
    from paper_1411_4356_gb300.workloads import batched_draws

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    params = sorted(batched_draws(512)[: args.systems], key=lambda p: -p.Nm)
    conc = args.concurrency if args.concurrency > 0 else 16
    for _ in range(args.warmup):
        sweep_pass(params, conc)
    clocks = ClockSampler(0)
    clocks.start()
    launches0 = api.kernel_launches()
    total = 0.0
    for _ in range(args.steps):
        dt, infos, rhos = sweep_pass(params, conc)
        total += dt
    launches = api.kernel_launches() - launches0
    clk = clocks.stop()
    line = {"metric": METRIC, "value": len(params) * args.steps / total, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 Krylov in FP64 refinement / TF32 no-jump products", "data": "synthetic",
            "config": {"workload": "sweep_6xNm_nojump", "systems": len(params), "Nc": 6,
                       "Nm": sorted({p.Nm for p in params}), "concurrency": conc, "restart": RESTART, "tol": 1e-12,
                       "eigendecomposition": "complex64",
                       "timed": "whole path per system (assembly, K + geev, GMRES, normalisation)"},
            "sweep": sweep_summary(params, infos, rhos), "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batched":
        run_batched(a)
    elif a.workload == "sweep":
        run_sweep(a)
    else:
        run_omss(a)
