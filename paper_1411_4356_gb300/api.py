"""Python binding of the omss C ABI (argument marshalling only).

Every step of the solve runs in libomss.so; PyTorch supplies CUDA device
memory and the current stream.  Names follow include/omss.h without the
``om_`` prefix.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import check, om_build_opts, om_params, om_solve_info, om_solve_opts
from .workloads import SystemParams

TRACE_MODES = {"replace": 0, "add": 1}


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _require_cuda(t: torch.Tensor, dtype, numel: int, name: str):
    if not t.is_cuda or t.dtype != dtype or t.numel() != numel or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor with {numel} elements")


# ---------------------------------------------------------------- allocator
_hook = None  # keeps the ctypes callbacks alive while they are installed


def _torch_alloc(nbytes, stream, ctx):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:  # noqa: BLE001 -- the library turns NULL into OM_ENOMEM
        return None


def _torch_free(ptr, stream, ctx):
    torch.cuda.caching_allocator_delete(int(ptr))


def set_allocator(alloc=None, free=None) -> None:
    """Route the library's device allocations through alloc(nbytes, stream, ctx) -> int
    and free(ptr, stream, ctx) (om_set_allocator); no arguments restores cudaMallocAsync."""
    global _hook
    lib = _lib.load()
    if alloc is None:
        check(lib.om_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None), "om_set_allocator")
        _hook = None
        return
    hook = (_lib.ALLOC_FN(alloc), _lib.FREE_FN(free))
    check(lib.om_set_allocator(hook[0], hook[1], None), "om_set_allocator")
    _hook = hook


def use_torch_allocator(on: bool = True) -> None:
    """Take the library's device memory from PyTorch's caching allocator (so that
    factors and Krylov bases are counted in torch.cuda.memory_allocated)."""
    if on:
        set_allocator(_torch_alloc, _torch_free)
    else:
        set_allocator()


def allocator_hook_calls() -> int:
    return int(_lib.load().om_allocator_hook_calls())


def to_om_params(p: SystemParams) -> om_params:
    return om_params(p.Nc, p.Nm, p.omega_m, p.Delta, p.kappa, p.g0, p.E, p.Q_m, p.n_th, p.g2, p.lam)


class Matrix:
    """Device CSR handle (om_matrix)."""

    def __init__(self, handle: int, params: SystemParams):
        self._h = ctypes.c_void_p(handle)
        self.params = params
        lib = _lib.load()
        N, nnz, w, ninf = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        check(lib.om_matrix_info(self._h, ctypes.byref(N), ctypes.byref(nnz), ctypes.byref(w), ctypes.byref(ninf)),
              "om_matrix_info")
        self.N, self.nnz, self.w, self.norm_inf = N.value, nnz.value, w.value, ninf.value

    @property
    def handle(self):
        return self._h

    def export(self, stream=None):
        """(rowptr int64, col int32, val complex128) numpy copies."""
        rp = np.empty(self.N + 1, dtype=np.int64)
        ci = np.empty(self.nnz, dtype=np.int32)
        va = np.empty(self.nnz, dtype=np.complex128)
        check(_lib.load().om_matrix_export(self._h, rp.ctypes.data_as(ctypes.c_void_p),
                                           ci.ctypes.data_as(ctypes.c_void_p), va.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.c_void_p(_stream(stream))), "om_matrix_export")
        return rp, ci, va

    def free(self):
        if self._h:
            _lib.load().om_matrix_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class ILU:
    """ILU factors handle (om_ilu)."""

    def __init__(self, handle: int, nnz_a: int, N: int = 0):
        self._h = ctypes.c_void_p(handle)
        self.N = N
        vals = [ctypes.c_int64() for _ in range(5)]
        check(_lib.load().om_ilu_info(self._h, *[ctypes.byref(v) for v in vals]), "om_ilu_info")
        self.nnz_l, self.nnz_u, self.n_guarded, self.levels_l, self.levels_u = (v.value for v in vals)
        self.fill = (self.nnz_l + self.nnz_u) / nnz_a
        t = (ctypes.c_double * 4)()
        check(_lib.load().om_ilu_timings(self._h, t), "om_ilu_timings")
        # host seconds: copy of A to the host, ILUT, dependency depths, tiled layout + upload
        self.timings = dict(zip(("copy", "ilut", "depth", "layout"), list(t)))

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            _lib.load().om_ilu_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_liouvillian(params: SystemParams, trace_mode: str = "replace", nth_floor: float = 1e-15,
                      stream=None) -> Matrix:
    """Eq. 1-5: trace-augmented Liouvillian on the device."""
    lib = _lib.load()
    out = ctypes.c_void_p()
    p = to_om_params(params)
    o = om_build_opts(TRACE_MODES[trace_mode], nth_floor)
    check(lib.om_build_liouvillian(ctypes.byref(p), ctypes.byref(o), ctypes.c_void_p(_stream(stream)),
                                   ctypes.byref(out)), "om_build_liouvillian")
    return Matrix(out.value, params)


def permute(A: Matrix, device_order: bool = True, stream=None):
    """Sec. III: (A_rcm, perm) with perm[new] = old as a CUDA int32 tensor; the
    RCM order is computed on the GPU, or with device_order=False by the serial
    walk on the host (the same permutation; om_permute_ex)."""
    lib = _lib.load()
    perm = torch.empty(A.N, dtype=torch.int32, device="cuda")
    out = ctypes.c_void_p()
    check(lib.om_permute_ex(A.handle, 1 if device_order else 0, ctypes.c_void_p(_stream(stream)), _ptr(perm),
                            ctypes.byref(out)), "om_permute")
    return Matrix(out.value, A.params), perm


def ilu_factor(A: Matrix, droptol: float, fill: float, compensate: bool = False, adjoint: bool = False,
               fp64_sweeps: bool = False, equilibrate: bool = False, permtol: float = 0.0, cap: str = "row",
               stream=None) -> ILU:
    """Sec. II: ILUT(droptol, fill) of a permuted matrix; adjoint=True also keeps
    the conjugate-transposed factors for the adjoint sweeps, fp64_sweeps=True
    the complex128 sweep data, equilibrate=True factors diag(r) A diag(c)
    (row, then column equilibration), permtol > 0 adds threshold column
    pivoting (ILUTP, om_ilutp_factor); cap="total" reads the fill cap as a
    running total NNZ(L) + NNZ(U) <= fill * NNZ(A) (flag 16) instead of a cap
    per row."""
    if cap not in ("row", "total"):
        raise ValueError(cap)
    lib = _lib.load()
    out = ctypes.c_void_p()
    flags = ((1 if compensate else 0) | (2 if adjoint else 0) | (4 if fp64_sweeps else 0)
             | (8 if equilibrate else 0) | (16 if cap == "total" else 0))
    if permtol != 0:
        check(lib.om_ilutp_factor(A.handle, float(droptol), float(fill), float(permtol), flags,
                                  ctypes.c_void_p(_stream(stream)), ctypes.byref(out)), "om_ilutp_factor")
    else:
        check(lib.om_ilu_factor(A.handle, float(droptol), float(fill), flags,
                                ctypes.c_void_p(_stream(stream)), ctypes.byref(out)), "om_ilu_factor")
    return ILU(out.value, A.nnz, A.N)


def liouvillian_row_host(params: SystemParams, k: int, nth_floor: float = 1e-15):
    """Row k of L from the assembly's closed form, on the host (om_liouvillian_row_host):
    (columns int64, values complex128) as numpy arrays."""
    cols = np.empty(32, dtype=np.int64)
    vals = np.empty(32, dtype=np.complex128)
    cnt = ctypes.c_int32()
    p = to_om_params(params)
    o = om_build_opts(0, nth_floor)
    check(_lib.load().om_liouvillian_row_host(ctypes.byref(p), ctypes.byref(o), int(k),
                                              cols.ctypes.data_as(ctypes.c_void_p),
                                              vals.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)),
          "om_liouvillian_row_host")
    return cols[:cnt.value].copy(), vals[:cnt.value].copy()


def rcm_order_host(rowptr, col):
    """The serial RCM order of the pattern of A + A^T on numpy CSR arrays, no
    device involved (om_rcm_order_host): perm[new] = old."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    perm = np.empty(len(rp) - 1, dtype=np.int32)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    check(_lib.load().om_rcm_order_host(len(rp) - 1, vp(rp), vp(ci), vp(perm)), "om_rcm_order_host")
    return perm


def ilu_factor_host(rowptr, col, val, droptol: float, fill: float, permtol: float = 0.0, compensate: bool = False,
                    equilibrate: bool = False, cap: str = "row") -> dict:
    """The host factorisation of ilu_factor alone, on numpy CSR arrays, no
    device involved (om_ilu_factor_host): a dict of numpy arrays (lp, li, lx,
    up, ui, ux -- strict parts in position space --, diag, q, r, c) and the
    counts n_guarded, n_swaps."""
    lib = _lib.load()
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.complex128)
    N = len(rp) - 1
    flags = (1 if compensate else 0) | (8 if equilibrate else 0) | (16 if cap == "total" else 0)
    h = ctypes.c_void_p()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    check(lib.om_ilu_factor_host(N, vp(rp), vp(ci), vp(va), float(droptol), float(fill), float(permtol), flags,
                                 ctypes.byref(h)), "om_ilu_factor_host")
    try:
        cnt = [ctypes.c_int64() for _ in range(4)]
        check(lib.om_host_ilu_sizes(h, *[ctypes.byref(x) for x in cnt]), "om_host_ilu_sizes")
        nl, nu, ng, ns = (x.value for x in cnt)
        out = dict(lp=np.empty(N + 1, np.int64), li=np.empty(nl, np.int32), lx=np.empty(nl, np.complex128),
                   up=np.empty(N + 1, np.int64), ui=np.empty(nu, np.int32), ux=np.empty(nu, np.complex128),
                   diag=np.empty(N, np.complex128), q=np.empty(N, np.int32), r=np.empty(N), c=np.empty(N))
        check(lib.om_host_ilu_export(h, *[vp(out[k]) for k in ("lp", "li", "lx", "up", "ui", "ux", "diag", "q",
                                                                "r", "c")]), "om_host_ilu_export")
    finally:
        lib.om_host_ilu_free(h)
    out["n_guarded"], out["n_swaps"] = ng, ns
    return out


def ilu_pivots(M: ILU, stream=None):
    """(pivoted, number of column swaps, q as a numpy int32 array: the column at each position)."""
    piv = ctypes.c_int32()
    ns = ctypes.c_int64()
    q = np.empty(M.N, dtype=np.int32)
    check(_lib.load().om_ilu_pivots(M.handle, ctypes.byref(piv), ctypes.byref(ns),
                                    q.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(_stream(stream))),
          "om_ilu_pivots")
    return bool(piv.value), int(ns.value), q


@dataclass
class SolveInfo:
    iterations: int
    cycles: int
    eta: float
    trace_before: float
    seconds: float
    residual_history: list
    status: int


def _opts(restart, max_iters, tol, precision, wait_timeout_ns, precond_fp64=False):
    return om_solve_opts(int(restart), int(max_iters), int(precision), 1 if precond_fp64 else 0, float(tol),
                         int(wait_timeout_ns))


def steady_state_solve(A_rcm: Matrix, M: ILU, perm: torch.Tensor, restart: int = 30, max_iters: int = 5000,
                       tol: float = 1e-10, precision: int = 0, x0: torch.Tensor | None = None,
                       wait_timeout_ns: int = 0, stream=None, raise_on_noconv: bool = True,
                       rho_out: torch.Tensor | None = None, precond_fp64: bool = False):
    """Sec. IV: rho (n x n complex128 CUDA tensor, rho[i, j] = rho_ij) and SolveInfo."""
    lib = _lib.load()
    n = A_rcm.params.Nc * A_rcm.params.Nm
    _require_cuda(perm, torch.int32, A_rcm.N, "perm")
    flat = rho_out if rho_out is not None else torch.empty(n * n, dtype=torch.complex128, device="cuda")
    _require_cuda(flat, torch.complex128, n * n, "rho_out")
    if x0 is not None:
        _require_cuda(x0, torch.complex128, A_rcm.N, "x0")
    o = _opts(restart, max_iters, tol, precision, wait_timeout_ns, precond_fp64)
    info = om_solve_info()
    st = lib.om_steady_state_solve(A_rcm.handle, M.handle, _ptr(perm), ctypes.byref(o), _ptr(x0), _ptr(flat),
                                   ctypes.byref(info), ctypes.c_void_p(_stream(stream)))
    si = SolveInfo(info.iterations, info.cycles, info.eta, info.trace_before, info.seconds,
                   list(info.residual_history[:min(info.cycles, 64)]), st)
    if st != 0 and not (st == -5 and not raise_on_noconv):
        check(st, "om_steady_state_solve")
    return flat.view(n, n).t(), si


def steady_state_adjoint(A_rcm: Matrix, M: ILU, perm: torch.Tensor, rho: torch.Tensor, grad_rho: torch.Tensor,
                         restart: int = 30, max_iters: int = 5000, tol: float = 1e-12, wait_timeout_ns: int = 0,
                         precond_fp64: bool = False, stream=None):
    """dF/d(Delta, E, g0, kappa) for a real loss with grad_rho = dF/dRe(rho) + i dF/dIm(rho)."""
    lib = _lib.load()
    n = A_rcm.params.Nc * A_rcm.params.Nm
    rho_flat = rho.t().contiguous().view(-1) if rho.dim() == 2 else rho
    g_flat = grad_rho.t().contiguous().view(-1) if grad_rho.dim() == 2 else grad_rho.contiguous()
    _require_cuda(rho_flat, torch.complex128, n * n, "rho")
    _require_cuda(g_flat, torch.complex128, n * n, "grad_rho")
    o = _opts(restart, max_iters, tol, 0, wait_timeout_ns, precond_fp64)
    p = to_om_params(A_rcm.params)
    out = (ctypes.c_double * 4)()
    info = om_solve_info()
    check(lib.om_steady_state_adjoint(A_rcm.handle, M.handle, _ptr(perm), ctypes.byref(o), ctypes.byref(p),
                                      _ptr(rho_flat), _ptr(g_flat), ctypes.byref(out), ctypes.byref(info),
                                      ctypes.c_void_p(_stream(stream))), "om_steady_state_adjoint")
    return list(out), SolveInfo(info.iterations, info.cycles, info.eta, info.trace_before, info.seconds,
                                list(info.residual_history[:min(info.cycles, 64)]), 0)


class NoJump:
    """Inverse of the no-jump part of Eq. 3 (om_nojump): the second preconditioner."""

    def __init__(self, handle: int, params: SystemParams):
        self._h = ctypes.c_void_p(handle)
        self.params = params
        n, tc, dmin = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        secs = (ctypes.c_double * 3)()
        check(_lib.load().om_nojump_info(self._h, ctypes.byref(n), ctypes.byref(tc), ctypes.byref(dmin), secs),
              "om_nojump_info")
        self.n, self.tensor_cores, self.min_abs_d = n.value, bool(tc.value), dmin.value
        # host seconds: K and its eigendecomposition, V^{-1}, operand layout
        self.timings = dict(zip(("eig", "inverse", "layout"), list(secs)))

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            _lib.load().om_nojump_free(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def nojump_factor(params: SystemParams, nth_floor: float = 1e-15, adjoint: bool = False, simt: bool = False,
                  eig32: bool = False, stream=None) -> NoJump:
    """K = -i H - (1/2) sum gamma O^dag O and its eigendecomposition (om_nojump_factor);
    adjoint=True keeps the operands of S^{-H}, simt=True selects complex64 SIMT products,
    eig32=True computes the eigendecomposition in complex64."""
    lib = _lib.load()
    out = ctypes.c_void_p()
    p = to_om_params(params)
    o = om_build_opts(0, nth_floor)
    flags = (1 if adjoint else 0) | (2 if simt else 0) | (4 if eig32 else 0)
    check(lib.om_nojump_factor(ctypes.byref(p), ctypes.byref(o), flags, ctypes.c_void_p(_stream(stream)),
                               ctypes.byref(out)), "om_nojump_factor")
    return NoJump(out.value, params)


def nojump_apply(M: NoJump, v: torch.Tensor, adjoint: bool = False, stream=None) -> torch.Tensor:
    """z = S^{-1} v (adjoint: S^{-H} v) for a CUDA complex128 vector of n*n entries."""
    _require_cuda(v, torch.complex128, M.n * M.n, "v")
    z = torch.empty_like(v)
    check(_lib.load().om_nojump_apply(M.handle, 2 if adjoint else 0, _ptr(v), _ptr(z),
                                      ctypes.c_void_p(_stream(stream))), "om_nojump_apply")
    return z


def steady_state_solve_nojump(A: Matrix, M: NoJump, restart: int = 50, max_iters: int = 5000, tol: float = 1e-10,
                              precision: int = 0, x0: torch.Tensor | None = None, stream=None,
                              raise_on_noconv: bool = True, rho_out: torch.Tensor | None = None,
                              wait_timeout_ns: int = 0):
    """Sec. IV's GMRES on the unpermuted L~ with the no-jump preconditioner:
    rho (n x n complex128 CUDA tensor) and SolveInfo."""
    lib = _lib.load()
    n = A.params.Nc * A.params.Nm
    flat = rho_out if rho_out is not None else torch.empty(n * n, dtype=torch.complex128, device="cuda")
    _require_cuda(flat, torch.complex128, n * n, "rho_out")
    if x0 is not None:
        _require_cuda(x0, torch.complex128, A.N, "x0")
    o = _opts(restart, max_iters, tol, precision, wait_timeout_ns)
    info = om_solve_info()
    st = lib.om_steady_state_solve_nojump(A.handle, M.handle, ctypes.byref(o), _ptr(x0), _ptr(flat),
                                          ctypes.byref(info), ctypes.c_void_p(_stream(stream)))
    si = SolveInfo(info.iterations, info.cycles, info.eta, info.trace_before, info.seconds,
                   list(info.residual_history[:min(info.cycles, 64)]), st)
    if st != 0 and not (st == -5 and not raise_on_noconv):
        check(st, "om_steady_state_solve_nojump")
    return flat.view(n, n).t(), si


def steady_state_adjoint_nojump(A: Matrix, M: NoJump, rho: torch.Tensor, grad_rho: torch.Tensor, restart: int = 50,
                                max_iters: int = 5000, tol: float = 1e-12, stream=None):
    """dF/d(Delta, E, g0, kappa) with the no-jump preconditioner (S^{-H})."""
    lib = _lib.load()
    n = A.params.Nc * A.params.Nm
    rho_flat = rho.t().contiguous().view(-1) if rho.dim() == 2 else rho
    g_flat = grad_rho.t().contiguous().view(-1) if grad_rho.dim() == 2 else grad_rho.contiguous()
    _require_cuda(rho_flat, torch.complex128, n * n, "rho")
    _require_cuda(g_flat, torch.complex128, n * n, "grad_rho")
    o = _opts(restart, max_iters, tol, 0, 0)
    p = to_om_params(A.params)
    out = (ctypes.c_double * 4)()
    info = om_solve_info()
    check(lib.om_steady_state_adjoint_nojump(A.handle, M.handle, ctypes.byref(o), ctypes.byref(p), _ptr(rho_flat),
                                             _ptr(g_flat), ctypes.byref(out), ctypes.byref(info),
                                             ctypes.c_void_p(_stream(stream))), "om_steady_state_adjoint_nojump")
    return list(out), SolveInfo(info.iterations, info.cycles, info.eta, info.trace_before, info.seconds,
                                list(info.residual_history[:min(info.cycles, 64)]), 0)


def spmv(A: Matrix, x: torch.Tensor, stream=None) -> torch.Tensor:
    _require_cuda(x, torch.complex128, A.N, "x")
    y = torch.empty_like(x)
    check(_lib.load().om_spmv(A.handle, _ptr(x), _ptr(y), ctypes.c_void_p(_stream(stream))), "om_spmv")
    return y


def liouvillian_apply(A: Matrix, x: torch.Tensor, stream=None) -> torch.Tensor:
    """y = L~ x from the stencil of Eq. 3 (unpermuted matrices only)."""
    _require_cuda(x, torch.complex128, A.N, "x")
    y = torch.empty_like(x)
    check(_lib.load().om_liouvillian_apply(A.handle, _ptr(x), _ptr(y), ctypes.c_void_p(_stream(stream))),
          "om_liouvillian_apply")
    return y


def ilu_apply(M: ILU, v: torch.Tensor, conj_transpose: bool = False, fp64: bool = False,
              single_block: bool = False, stream=None) -> torch.Tensor:
    """z = M^{-1} v (or M^{-H} v), M = L U, or diag(r)^{-1} L U diag(c)^{-1} for
    equilibrated factors; fp64 selects the complex128 sweeps, single_block
    keeps the complex64 sweeps in one thread block."""
    z = torch.empty_like(v)
    flags = (1 if fp64 else 0) | (2 if conj_transpose else 0) | (4 if single_block else 0)
    check(_lib.load().om_ilu_apply(M.handle, flags, _ptr(v.contiguous()), _ptr(z),
                                   ctypes.c_void_p(_stream(stream))), "om_ilu_apply")
    return z


def ilu_condest(M: ILU, fp64: bool = False, single_block: bool = False, stream=None) -> float:
    """||M^{-1} e||_inf, e = ones (Sec. IV's stability estimate of the factors)."""
    out = ctypes.c_double()
    flags = (1 if fp64 else 0) | (4 if single_block else 0)
    check(_lib.load().om_ilu_condest(M.handle, flags, ctypes.byref(out), ctypes.c_void_p(_stream(stream))),
          "om_ilu_condest")
    return out.value


def observables(Nc: int, Nm: int, rho: torch.Tensor, stream=None):
    """(<a^dag a>, <b^dag b>) of a CUDA rho."""
    flat = rho.t().contiguous().view(-1) if rho.dim() == 2 else rho
    out = (ctypes.c_double * 2)()
    check(_lib.load().om_observables(int(Nc), int(Nm), _ptr(flat), ctypes.byref(out),
                                     ctypes.c_void_p(_stream(stream))), "om_observables")
    return out[0], out[1]


def steady_state_sweep_nojump(params_list, restart: int = 50, max_iters: int = 5000, tol: float = 1e-12,
                              precision: int = 0, trace_mode: str = "replace", nth_floor: float = 1e-15,
                              eig32: bool = False, simt: bool = False, concurrency: int = 8, stream=None):
    """The whole no-jump path for many parameter sets on concurrent streams
    (om_steady_state_sweep_nojump).  Returns ([rho n x n CUDA tensors], [SolveInfo])."""
    lib = _lib.load()
    count = len(params_list)
    P = (om_params * max(count, 1))(*[to_om_params(p) for p in params_list])
    rhos = [torch.empty(p.n * p.n, dtype=torch.complex128, device="cuda") for p in params_list]
    Rh = (ctypes.c_void_p * max(count, 1))(*[r.data_ptr() for r in rhos])
    infos = (om_solve_info * max(count, 1))()
    status = (ctypes.c_int32 * max(count, 1))()
    o = _opts(restart, max_iters, tol, precision, 0)
    b = om_build_opts(TRACE_MODES[trace_mode], nth_floor)
    flags = (2 if simt else 0) | (4 if eig32 else 0)
    check(lib.om_steady_state_sweep_nojump(count, ctypes.cast(P, ctypes.c_void_p), ctypes.byref(b), flags,
                                           ctypes.byref(o), ctypes.cast(Rh, ctypes.c_void_p),
                                           ctypes.cast(infos, ctypes.c_void_p), ctypes.cast(status, ctypes.c_void_p),
                                           int(concurrency), ctypes.c_void_p(_stream(stream))),
          "om_steady_state_sweep_nojump")
    out_rho, out_info = [], []
    for i, p in enumerate(params_list):
        out_rho.append(rhos[i].view(p.n, p.n).t())
        inf = infos[i]
        out_info.append(SolveInfo(inf.iterations, inf.cycles, inf.eta, inf.trace_before, inf.seconds,
                                  list(inf.residual_history[:min(inf.cycles, 64)]), int(status[i])))
    return out_rho, out_info


def phonon_distribution(Nc: int, Nm: int, rho: torch.Tensor, stream=None):
    """(P[m] numpy array, <N_b>, <N_b^2>, Fano factor) of a CUDA rho (Sec. V, Fig. 5)."""
    flat = rho.t().contiguous().view(-1) if rho.dim() == 2 else rho
    P = np.empty(int(Nm), dtype=np.float64)
    mom = (ctypes.c_double * 3)()
    check(_lib.load().om_phonon_distribution(int(Nc), int(Nm), _ptr(flat), P.ctypes.data_as(ctypes.c_void_p),
                                             ctypes.byref(mom), ctypes.c_void_p(_stream(stream))),
          "om_phonon_distribution")
    return P, mom[0], mom[1], mom[2]


def kernel_launches() -> int:
    """Kernels launched by libomss.so since it was loaded."""
    return int(_lib.load().om_kernel_launches())


PROF_SWEEP, PROF_SPMV, PROF_SPLIT, PROF_NOJUMP, PROF_KRYLOV, PROF_STENCIL = 0, 1, 2, 3, 4, 5


def profile(enable: bool) -> None:
    """Start (True) or stop (False) event timing of sweep and SpMV launches."""
    check(_lib.load().om_profile(1 if enable else 0), "om_profile")


def profile_read(category: int):
    """(total device milliseconds, launch count) recorded for a category."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    check(_lib.load().om_profile_read(int(category), ctypes.byref(ms), ctypes.byref(n)), "om_profile_read")
    return ms.value, n.value


THETA_NAMES = ("Delta", "E", "g0", "kappa")


class SteadyState(torch.autograd.Function):
    """rho_ss as a differentiable function of theta = (Delta, E, g0, kappa).

    forward(theta, base, options) builds, permutes and factors the
    Liouvillian at `base` with theta substituted, and returns rho (n x n,
    complex128, CUDA).  backward solves the adjoint equation
    L~^H mu = dF/drho with the same permuted ILU and returns
    dF/dtheta = -Re(mu^H dL~/dtheta rho) (om_steady_state_adjoint)."""

    @staticmethod
    def forward(ctx, theta, base: SystemParams, options: dict):
        vals = [float(v) for v in theta.detach().cpu().tolist()]
        p = base.with_(**dict(zip(THETA_NAMES, vals)))
        o = dict(options)
        A = build_liouvillian(p, o.get("trace_mode", "replace"), o.get("nth_floor", 1e-15))
        Ar, perm = permute(A)
        A.free()
        M = ilu_factor(Ar, o.get("droptol", 1e-4), o.get("fill", 10.0), adjoint=True)
        rho, info = steady_state_solve(Ar, M, perm, restart=o.get("restart", 30), tol=o.get("tol", 1e-12),
                                       max_iters=o.get("max_iters", 5000))
        rho = rho.contiguous()
        ctx.state = (Ar, M, perm, rho, o)
        ctx.theta_device = theta.device
        ctx.info = info
        return rho

    @staticmethod
    def backward(ctx, grad_rho):
        Ar, M, perm, rho, o = ctx.state
        g, _ = steady_state_adjoint(Ar, M, perm, rho, grad_rho.to(torch.complex128), restart=o.get("restart", 30),
                                    tol=o.get("adjoint_tol", 1e-12), max_iters=o.get("max_iters", 5000))
        return torch.tensor(g, dtype=torch.float64, device=ctx.theta_device), None, None


def steady_state(theta: torch.Tensor, base: SystemParams, **options) -> torch.Tensor:
    """Differentiable steady state: theta = (Delta, E, g0, kappa) (float64)."""
    return SteadyState.apply(theta, base, options)


def steady_state_solve_batched(systems, restart: int = 30, max_iters: int = 5000, tol: float = 1e-10,
                               precision: int = 0, concurrency: int = 0, stream=None):
    """Solve many (A_rcm, M, perm) systems together (om_steady_state_solve_batched).

    concurrency <= 0 runs the lock-step engine (one launch per kernel and
    Krylov step for all systems; precision 0 only); concurrency > 0 runs that
    many single solves at a time on their own streams.
    Returns ([rho n x n CUDA tensors], [SolveInfo])."""
    lib = _lib.load()
    count = len(systems)
    Ah = (ctypes.c_void_p * count)(*[A.handle.value for A, M, perm in systems])
    Mh = (ctypes.c_void_p * count)(*[M.handle.value for A, M, perm in systems])
    Ph = (ctypes.c_void_p * count)(*[perm.data_ptr() for A, M, perm in systems])
    rhos = [torch.empty(A.params.Nc * A.params.Nm * A.params.Nc * A.params.Nm, dtype=torch.complex128,
                        device="cuda") for A, M, perm in systems]
    Rh = (ctypes.c_void_p * count)(*[r.data_ptr() for r in rhos])
    infos = (om_solve_info * count)()
    status = (ctypes.c_int32 * count)()
    o = _opts(restart, max_iters, tol, precision, 0)
    check(lib.om_steady_state_solve_batched(count, Ah, Mh, Ph, ctypes.byref(o), Rh, infos, status, int(concurrency),
                                            ctypes.c_void_p(_stream(stream))), "om_steady_state_solve_batched")
    out_rho, out_info = [], []
    for i, (A, M, perm) in enumerate(systems):
        n = A.params.Nc * A.params.Nm
        out_rho.append(rhos[i].view(n, n).t())
        inf = infos[i]
        out_info.append(SolveInfo(inf.iterations, inf.cycles, inf.eta, inf.trace_before, inf.seconds,
                                  list(inf.residual_history[:min(inf.cycles, 64)]), int(status[i])))
    return out_rho, out_info
