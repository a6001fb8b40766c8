"""Thin Python binding of libhzn (the C-ABI declared in include/hzn.h).

The functions ``hz_*`` below have the names, arguments and return codes of the C calls; they
only marshal arguments.  Device memory and streams come from PyTorch (``torch.empty`` on the
CUDA device, ``torch.cuda.current_stream()``); every step of the numerical method runs in the
library's CUDA kernels.  ``Solver`` bundles the calls for one grid.

The library is loaded on first use.  If it is missing or fails to load, ``lib()`` raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

HZ_OK, HZ_WARN_C2P = 0, 1
HZ_ERR_ARG, HZ_ERR_CUDA, HZ_ERR_STATE, HZ_ERR_WORKSPACE, HZ_ERR_UNSUPPORTED = -1, -2, -3, -4, -5
HZ_ERR_TOO_LARGE = -6
HZ_NOALLOC_SCRATCH_BYTES = 16 << 20
HZ_BC_OUTFLOW, HZ_BC_PERIODIC = 0, 1
HZ_FP64, HZ_MIXED, HZ_FP64_DW = 0, 1, 2
HZ_RECON_MC, HZ_RECON_PPM = 0, 1
HZ_C2P_2D, HZ_C2P_1D = 0, 1

EXPORTED = (
    "hz_workspace_bytes", "hz_create", "hz_destroy", "hz_set_metric", "hz_set_primitives",
    "hz_get_primitives", "hz_get_conserved", "hz_step", "hz_step_cfl", "hz_max_speed",
    "hz_get_stats", "hz_strerror", "hz_version", "hz_step_noalloc", "hz_dw_selftest",
    "hz_rcp_selftest", "hz_last_cuda_error", "hz_cuda_error_string",
)
HZ_DW_NRESULTS = 9


class hz_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("bc", ctypes.c_int * 3), ("dx", ctypes.c_double * 3)]


class hz_options(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("cleaning", ctypes.c_int),
        ("ch", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("rho_floor", ctypes.c_double),
        ("rho_atm", ctypes.c_double),
        ("p_floor", ctypes.c_double),
        ("atm_K", ctypes.c_double),
        ("c2p_maxit", ctypes.c_int),
        ("c2p_tol", ctypes.c_double),
        ("recon", ctypes.c_int),
        ("c2p", ctypes.c_int),
    ]


class hz_stats(ctypes.Structure):
    _fields_ = [
        ("c2p_failures", ctypes.c_longlong),
        ("c2p_max_iters", ctypes.c_int),
        ("max_speed", ctypes.c_double),
        ("t", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("steps", ctypes.c_longlong),
    ]


_lock = threading.Lock()
_lib = None


class HznError(RuntimeError):
    def __init__(self, code: int, call: str):
        msg = f"{call} failed: {code} ({hz_strerror(code)})"
        self.cuda_code = 0
        if code == HZ_ERR_CUDA:
            self.cuda_code = int(lib().hz_last_cuda_error())
            msg += f"; CUDA error {self.cuda_code}: {lib().hz_cuda_error_string(self.cuda_code).decode()}"
        super().__init__(msg)
        self.code = code


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libhzn.so (raises if it was not built; ``build.build_library()`` builds it)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libhzn.so is not built ({path}); run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            vp, dp = ctypes.c_void_p, P(ctypes.c_double)
            L.hz_workspace_bytes.argtypes = [P(hz_grid), P(hz_options), P(ctypes.c_size_t)]
            L.hz_create.argtypes = [P(vp), P(hz_grid), P(hz_options), vp, ctypes.c_size_t, vp]
            L.hz_destroy.argtypes = [vp]
            L.hz_set_metric.argtypes = [vp, vp]
            L.hz_set_primitives.argtypes = [vp, vp]
            L.hz_get_primitives.argtypes = [vp, vp]
            L.hz_get_conserved.argtypes = [vp, vp]
            L.hz_step.argtypes = [vp, ctypes.c_double]
            L.hz_step_cfl.argtypes = [vp, ctypes.c_double, ctypes.c_double]
            L.hz_max_speed.argtypes = [vp, dp]
            L.hz_get_stats.argtypes = [vp, P(hz_stats)]
            L.hz_step_noalloc.argtypes = [P(hz_grid), P(hz_options), vp, vp, vp, ctypes.c_double,
                                          ctypes.c_int, vp]
            L.hz_dw_selftest.argtypes = [vp, vp, vp, ctypes.c_longlong, vp]
            L.hz_rcp_selftest.argtypes = [vp, vp, ctypes.c_longlong, vp]
            L.hz_strerror.argtypes = [ctypes.c_int]
            L.hz_strerror.restype = ctypes.c_char_p
            L.hz_version.restype = ctypes.c_int
            L.hz_last_cuda_error.argtypes = []
            L.hz_cuda_error_string.argtypes = [ctypes.c_int]
            L.hz_cuda_error_string.restype = ctypes.c_char_p
            for name in EXPORTED:
                if name not in ("hz_strerror", "hz_version", "hz_cuda_error_string"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


# ------------------------------------------------------------------ C calls, same names
def hz_strerror(code: int) -> str:
    return lib().hz_strerror(int(code)).decode()


def hz_version() -> int:
    return int(lib().hz_version())


def hz_dw_selftest(a, b):
    """Double-word results of the HZ_FP64_DW arithmetic for the doubles a, b (1-D float64 CUDA
    tensors of one length n): a (HZ_DW_NRESULTS, 2, n) float64 tensor of (hi, lo) per result."""
    import torch

    n = int(a.numel())
    out = torch.empty((HZ_DW_NRESULTS, 2, n), dtype=torch.float64, device=a.device)
    st = torch.cuda.current_stream(a.device).cuda_stream
    _check(lib().hz_dw_selftest(a.data_ptr(), b.data_ptr(), out.data_ptr(), n, st), "hz_dw_selftest")
    return out


def hz_rcp_selftest(x):
    """The FP64 kernels' reciprocal of each element of x (a 1-D float64 CUDA tensor)."""
    import torch

    out = torch.empty_like(x)
    st = torch.cuda.current_stream(x.device).cuda_stream
    _check(lib().hz_rcp_selftest(x.data_ptr(), out.data_ptr(), int(x.numel()), st), "hz_rcp_selftest")
    return out


def hz_workspace_bytes(grid: hz_grid, opts: hz_options) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().hz_workspace_bytes(ctypes.byref(grid), ctypes.byref(opts), ctypes.byref(n)),
           "hz_workspace_bytes")
    return int(n.value)


def hz_create(grid: hz_grid, opts: hz_options, d_workspace: int, nbytes: int, stream: int) -> int:
    h = ctypes.c_void_p(0)
    _check(lib().hz_create(ctypes.byref(h), ctypes.byref(grid), ctypes.byref(opts),
                           ctypes.c_void_p(d_workspace), nbytes, ctypes.c_void_p(stream)), "hz_create")
    return int(h.value)


def hz_destroy(ctx: int) -> None:
    lib().hz_destroy(ctypes.c_void_p(ctx))


def hz_set_metric(ctx: int, d_metric: int) -> None:
    _check(lib().hz_set_metric(ctypes.c_void_p(ctx), ctypes.c_void_p(d_metric)), "hz_set_metric")


def hz_set_primitives(ctx: int, d_prim: int) -> None:
    _check(lib().hz_set_primitives(ctypes.c_void_p(ctx), ctypes.c_void_p(d_prim)), "hz_set_primitives")


def hz_get_primitives(ctx: int, d_prim: int) -> None:
    _check(lib().hz_get_primitives(ctypes.c_void_p(ctx), ctypes.c_void_p(d_prim)), "hz_get_primitives")


def hz_get_conserved(ctx: int, d_cons: int) -> None:
    _check(lib().hz_get_conserved(ctypes.c_void_p(ctx), ctypes.c_void_p(d_cons)), "hz_get_conserved")


def hz_step(ctx: int, dt: float) -> None:
    _check(lib().hz_step(ctypes.c_void_p(ctx), float(dt)), "hz_step")


def hz_step_cfl(ctx: int, cfl: float, t_end: float) -> None:
    _check(lib().hz_step_cfl(ctypes.c_void_p(ctx), float(cfl), float(t_end)), "hz_step_cfl")


def hz_max_speed(ctx: int) -> float:
    v = ctypes.c_double(0.0)
    _check(lib().hz_max_speed(ctypes.c_void_p(ctx), ctypes.byref(v)), "hz_max_speed")
    return float(v.value)


def hz_get_stats(ctx: int) -> hz_stats:
    s = hz_stats()
    code = lib().hz_get_stats(ctypes.c_void_p(ctx), ctypes.byref(s))
    if code < 0:
        raise HznError(code, "hz_get_stats")
    return s


def hz_step_noalloc(grid: hz_grid, opts: hz_options, d_metric: int, d_prim_in: int, d_prim_out: int,
                    dt: float, nsteps: int, stream: int) -> int:
    """nsteps fixed-dt RK3 steps with the library's static scratch (no allocation at all).
    Returns HZ_OK or HZ_WARN_C2P (failed recoveries reset to the atmosphere); the output is
    written when the call returns."""
    return _check(lib().hz_step_noalloc(ctypes.byref(grid), ctypes.byref(opts), ctypes.c_void_p(d_metric),
                                 ctypes.c_void_p(d_prim_in), ctypes.c_void_p(d_prim_out), float(dt),
                                 int(nsteps), ctypes.c_void_p(stream)), "hz_step_noalloc")


def _check(code: int, call: str) -> int:
    if code < 0:
        raise HznError(code, call)
    return code


# ------------------------------------------------------------------ convenience
def make_grid(n, dx, bc) -> hz_grid:
    g = hz_grid()
    for d in range(3):
        g.n[d], g.dx[d], g.bc[d] = int(n[d]), float(dx[d]), int(bc[d])
    return g


def make_options(gamma: float, precision: int = HZ_FP64, cleaning: bool = False, ch: float = 0.0,
                 kappa: float = 0.0, rho_floor: float = 1e-12, rho_atm: float = 0.0,
                 p_floor: float = 1e-14, atm_K: float = 0.0, c2p_maxit: int = 50,
                 c2p_tol: float = 1e-12, recon: int = HZ_RECON_MC, c2p: int = HZ_C2P_2D) -> hz_options:
    return hz_options(float(gamma), int(precision), int(bool(cleaning)), float(ch), float(kappa),
                      float(rho_floor), float(rho_atm), float(p_floor), float(atm_K), int(c2p_maxit),
                      float(c2p_tol), int(recon), int(c2p))


class Solver:
    """One grid on the current CUDA device: workspace from torch, calls through the C-ABI."""

    def __init__(self, n, dx, bc, options: hz_options, device: Optional[str] = None, stream=None):
        import torch

        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.n = tuple(int(k) for k in n)
        self.grid = make_grid(n, dx, bc)
        self.options = options
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = hz_workspace_bytes(self.grid, options)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.ctx = hz_create(self.grid, options, aligned, nbytes, self.stream.cuda_stream)
        self.ghost = tuple(1 if k > 1 else 0 for k in self.n)

    @classmethod
    def for_problem(cls, prob, precision: int = HZ_FP64, c2p_maxit: int = 50, c2p_tol: float = 1e-12,
                    **kw):
        opts = make_options(prob.gamma, precision=precision, cleaning=prob.cleaning, ch=prob.ch,
                            kappa=prob.kappa, rho_floor=prob.rho_floor, rho_atm=prob.rho_atm,
                            p_floor=prob.p_floor, atm_K=prob.atm_K, c2p_maxit=c2p_maxit,
                            c2p_tol=c2p_tol, recon=prob.recon, c2p=prob.c2p)
        s = cls(prob.n, prob.dx, prob.bc, opts, **kw)
        s.set_metric(prob.metric)
        s.set_primitives(prob.prim)
        return s

    def close(self):
        if getattr(self, "ctx", None):
            hz_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a):
        t = self.torch
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        a = a.to(device=self.device, dtype=t.float64).contiguous()
        return a

    def _shape(self):
        return (9, self.n[2], self.n[1], self.n[0])

    def set_metric(self, metric):
        m = self._dev(metric)
        g = self.ghost
        want = (10, self.n[2] + 2 * g[2], self.n[1] + 2 * g[1], self.n[0] + 2 * g[0])
        if tuple(m.shape) != want:
            raise ValueError(f"metric shape {tuple(m.shape)} != {want}")
        hz_set_metric(self.ctx, m.data_ptr())
        self._keep = m  # keep alive until the copy has run on the stream

    def set_primitives(self, prim):
        p = self._dev(prim)
        if tuple(p.shape) != self._shape():
            raise ValueError(f"primitive shape {tuple(p.shape)} != {self._shape()}")
        hz_set_primitives(self.ctx, p.data_ptr())
        self._keep_p = p

    def step(self, dt: float):
        hz_step(self.ctx, dt)

    def step_cfl(self, cfl: float, t_end: float):
        """One RK3 step of dt = cfl / max_speed(), taken on the device, clipped at t_end."""
        hz_step_cfl(self.ctx, cfl, t_end)

    def max_speed(self) -> float:
        """CFL rate of the current state: max over cells of sum_d max|lambda_d| / dx_d."""
        return hz_max_speed(self.ctx)

    def stats(self) -> hz_stats:
        return hz_get_stats(self.ctx)

    def primitives(self):
        out = self.torch.empty(self._shape(), dtype=self.torch.float64, device=self.device)
        hz_get_primitives(self.ctx, out.data_ptr())
        return out

    def conserved(self):
        out = self.torch.empty(self._shape(), dtype=self.torch.float64, device=self.device)
        hz_get_conserved(self.ctx, out.data_ptr())
        return out

    def evolve(self, t_end: float, cfl: float, max_steps: int = 1 << 40) -> int:
        """Advance with device-side CFL steps until t_end; returns the steps taken."""
        steps = 0
        while steps < max_steps:
            s = self.stats()
            if s.t >= t_end:
                break
            self.step_cfl(cfl, t_end)
            steps += 1
        return steps


# ------------------------------------------------------------------ ensembles of 1-D tubes
ENSEMBLE_EXPORTED = (
    "hz_ensemble_workspace_bytes", "hz_ensemble_create", "hz_ensemble_destroy",
    "hz_ensemble_set_primitives", "hz_ensemble_set_launch", "hz_ensemble_run",
    "hz_ensemble_get_primitives", "hz_ensemble_results", "hz_ensemble_autotune",
)


def _ens_lib():
    L = lib()
    if not getattr(L, "_ens_ready", False):
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        ip, dp, lp = P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_longlong)
        L.hz_ensemble_workspace_bytes.argtypes = [ctypes.c_int, ip, P(ctypes.c_size_t)]
        L.hz_ensemble_create.argtypes = [P(vp), ctypes.c_int, ip, dp, dp, P(hz_options), vp,
                                         ctypes.c_size_t, vp]
        L.hz_ensemble_destroy.argtypes = [vp]
        L.hz_ensemble_set_primitives.argtypes = [vp, vp]
        L.hz_ensemble_set_launch.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.hz_ensemble_run.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_longlong, ctypes.c_int]
        L.hz_ensemble_get_primitives.argtypes = [vp, vp]
        L.hz_ensemble_results.argtypes = [vp, dp, lp, lp]
        L.hz_ensemble_autotune.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ip, ip,
                                           P(ctypes.c_float)]
        for name in ENSEMBLE_EXPORTED:
            getattr(L, name).restype = ctypes.c_int
        L._ens_ready = True
    return L


def _iarr(x):
    a = np.ascontiguousarray(x, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _darr(x):
    a = np.ascontiguousarray(x, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def hz_ensemble_workspace_bytes(n) -> int:
    na, np_ = _iarr(n)
    out = ctypes.c_size_t(0)
    _check(_ens_lib().hz_ensemble_workspace_bytes(len(na), np_, ctypes.byref(out)),
           "hz_ensemble_workspace_bytes")
    return int(out.value)


def hz_ensemble_create(n, dx, gamma, opts: hz_options, d_workspace: int, nbytes: int, stream: int) -> int:
    na, np_ = _iarr(n)
    da, dp_ = _darr(dx)
    ga, gp = _darr(gamma)
    h = ctypes.c_void_p(0)
    _check(_ens_lib().hz_ensemble_create(ctypes.byref(h), len(na), np_, dp_, gp, ctypes.byref(opts),
                                         ctypes.c_void_p(d_workspace), nbytes, ctypes.c_void_p(stream)),
           "hz_ensemble_create")
    return int(h.value)


def hz_ensemble_destroy(ens: int) -> None:
    _ens_lib().hz_ensemble_destroy(ctypes.c_void_p(ens))


def hz_ensemble_set_primitives(ens: int, d_prim: int) -> None:
    _check(_ens_lib().hz_ensemble_set_primitives(ctypes.c_void_p(ens), ctypes.c_void_p(d_prim)),
           "hz_ensemble_set_primitives")


def hz_ensemble_set_launch(ens: int, threads: int, ctas_per_sm: int) -> None:
    _check(_ens_lib().hz_ensemble_set_launch(ctypes.c_void_p(ens), int(threads), int(ctas_per_sm)),
           "hz_ensemble_set_launch")


def hz_ensemble_run(ens: int, t_end: float, cfl: float, max_steps: int = 1 << 40, use_graph: bool = False) -> None:
    _check(_ens_lib().hz_ensemble_run(ctypes.c_void_p(ens), float(t_end), float(cfl), int(max_steps),
                                      int(bool(use_graph))), "hz_ensemble_run")


def hz_ensemble_get_primitives(ens: int, d_prim: int) -> None:
    _check(_ens_lib().hz_ensemble_get_primitives(ctypes.c_void_p(ens), ctypes.c_void_p(d_prim)),
           "hz_ensemble_get_primitives")


def hz_ensemble_results(ens: int, ntubes: int):
    t = np.zeros(ntubes)
    st = np.zeros(ntubes, dtype=np.int64)
    fl = np.zeros(ntubes, dtype=np.int64)
    code = _ens_lib().hz_ensemble_results(ctypes.c_void_p(ens), t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          st.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                          fl.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    if code < 0:
        raise HznError(code, "hz_ensemble_results")
    return t, st, fl


def hz_ensemble_autotune(ens: int, d_prim: int, t_probe: float, cfl: float):
    th, cps = ctypes.c_int(0), ctypes.c_int(0)
    ms = (ctypes.c_float * 5)()
    _check(_ens_lib().hz_ensemble_autotune(ctypes.c_void_p(ens), ctypes.c_void_p(d_prim), float(t_probe),
                                           float(cfl), ctypes.byref(th), ctypes.byref(cps), ms),
           "hz_ensemble_autotune")
    return int(th.value), int(cps.value), list(ms)


class Ensemble:
    """Independent 1-D tubes (workloads.Problem instances along x) on the current CUDA device."""

    def __init__(self, problems, rho_floor: float = 1e-12, p_floor: float = 1e-14, c2p_maxit: int = 50,
                 c2p_tol: float = 1e-12, stream=None):
        import torch

        self.torch = torch
        self.problems = list(problems)
        self.n = np.array([p.n[0] for p in self.problems], dtype=np.int32)
        dx = np.array([p.dx[0] for p in self.problems])
        gam = np.array([p.gamma for p in self.problems])
        self.options = make_options(2.0, rho_floor=rho_floor, p_floor=p_floor, c2p_maxit=c2p_maxit,
                                    c2p_tol=c2p_tol)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        nbytes = hz_ensemble_workspace_bytes(self.n)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        self.ens = hz_ensemble_create(self.n, dx, gam, self.options, base, nbytes, self.stream.cuda_stream)
        self.ncat = int(self.n.sum())
        self.off = np.concatenate([[0], np.cumsum(self.n)[:-1]]).astype(np.int64)
        host = np.zeros((9, self.ncat))
        for p, o in zip(self.problems, self.off):
            host[:, o:o + p.n[0]] = p.prim[:, 0, 0, :]
        self.host_prim = host
        self.d_prim = torch.from_numpy(host).to("cuda")
        torch.cuda.synchronize()
        self.set_primitives()

    def close(self):
        if getattr(self, "ens", None):
            hz_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_primitives(self):
        with self.torch.cuda.stream(self.stream):
            hz_ensemble_set_primitives(self.ens, self.d_prim.data_ptr())

    def autotune(self, t_probe: float = 0.02, cfl: float = 0.5):
        return hz_ensemble_autotune(self.ens, self.d_prim.data_ptr(), t_probe, cfl)

    def run(self, t_end: float, cfl: float = 0.5, use_graph: bool = True, max_steps: int = 1 << 40):
        hz_ensemble_run(self.ens, t_end, cfl, max_steps, use_graph)

    def primitives(self):
        """List of (9, 1, 1, n) arrays, one per tube."""
        out = self.torch.empty((9, self.ncat), dtype=self.torch.float64, device="cuda")
        hz_ensemble_get_primitives(self.ens, out.data_ptr())
        self.stream.synchronize()
        h = out.cpu().numpy()
        return [h[:, o:o + n].reshape(9, 1, 1, n).copy() for o, n in zip(self.off, self.n)]

    def results(self):
        return hz_ensemble_results(self.ens, len(self.n))


# ------------------------------------------------------------------ adjoint of a fixed-step run
ADJOINT_EXPORTED = (
    "hz_adjoint_workspace_bytes", "hz_adjoint_create", "hz_adjoint_destroy",
    "hz_adjoint_checkpoint_interval", "hz_adjoint_forward", "hz_adjoint_backward",
)


def _adj_lib():
    L = lib()
    if not getattr(L, "_adj_ready", False):
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        ip = P(ctypes.c_int)
        L.hz_adjoint_workspace_bytes.argtypes = [P(hz_grid), P(hz_options), ctypes.c_int, ctypes.c_int,
                                                 P(ctypes.c_size_t)]
        L.hz_adjoint_create.argtypes = [P(vp), vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp,
                                        ctypes.c_size_t]
        L.hz_adjoint_destroy.argtypes = [vp]
        L.hz_adjoint_checkpoint_interval.argtypes = [vp, ip, ip]
        L.hz_adjoint_forward.argtypes = [vp, vp, vp]
        L.hz_adjoint_backward.argtypes = [vp, vp, vp, vp]
        for name in ADJOINT_EXPORTED:
            getattr(L, name).restype = ctypes.c_int
        L._adj_ready = True
    return L


def hz_adjoint_workspace_bytes(grid: hz_grid, opts: hz_options, nsteps: int, ckpt_every: int = 0) -> int:
    n = ctypes.c_size_t(0)
    _check(_adj_lib().hz_adjoint_workspace_bytes(ctypes.byref(grid), ctypes.byref(opts), int(nsteps),
                                                 int(ckpt_every), ctypes.byref(n)),
           "hz_adjoint_workspace_bytes")
    return int(n.value)


def hz_adjoint_create(ctx: int, nsteps: int, dt: float, ckpt_every: int, d_workspace: int, nbytes: int) -> int:
    h = ctypes.c_void_p(0)
    _check(_adj_lib().hz_adjoint_create(ctypes.byref(h), ctx, int(nsteps), float(dt), int(ckpt_every),
                                        d_workspace, nbytes), "hz_adjoint_create")
    return h.value


def hz_adjoint_destroy(adj: int) -> None:
    _check(_adj_lib().hz_adjoint_destroy(adj), "hz_adjoint_destroy")


def hz_adjoint_checkpoint_interval(adj: int):
    every, segs = ctypes.c_int(0), ctypes.c_int(0)
    _check(_adj_lib().hz_adjoint_checkpoint_interval(adj, ctypes.byref(every), ctypes.byref(segs)),
           "hz_adjoint_checkpoint_interval")
    return int(every.value), int(segs.value)


def hz_adjoint_forward(adj: int, d_prim_in: int, d_prim_out: int) -> None:
    _check(_adj_lib().hz_adjoint_forward(adj, d_prim_in, d_prim_out), "hz_adjoint_forward")


def hz_adjoint_backward(adj: int, d_gprim_out: int, d_gcons_out: Optional[int], d_gprim_in: int) -> None:
    _check(_adj_lib().hz_adjoint_backward(adj, d_gprim_out, d_gcons_out, d_gprim_in), "hz_adjoint_backward")


class Adjoint:
    """Reverse-mode gradient of ``nsteps`` fixed steps of size ``dt`` on a Solver's grid.

    ``forward(prim0)`` runs the steps (storing sqrt(n) checkpoints) and returns the final
    primitives; ``backward(gprim)`` returns dJ/dP(0) for dJ/dP(n) = gprim.  ``evolve(prim0)`` is
    the same pair as a differentiable torch operation (torch.autograd.Function)."""

    def __init__(self, solver: Solver, nsteps: int, dt: float, ckpt_every: int = 0):
        t = solver.torch
        self.torch = t
        self.solver = solver
        self.nsteps = int(nsteps)
        self.dt = float(dt)
        nbytes = hz_adjoint_workspace_bytes(solver.grid, solver.options, nsteps, ckpt_every)
        self.workspace = t.empty(nbytes + 256, dtype=t.uint8, device=solver.device)
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        self.adj = hz_adjoint_create(solver.ctx, nsteps, dt, ckpt_every, base, nbytes)
        self.checkpoint_every, self.segments = hz_adjoint_checkpoint_interval(self.adj)
        self.generation = 0

    def close(self):
        if getattr(self, "adj", None):
            hz_adjoint_destroy(self.adj)
            self.adj = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, prim0):
        s = self.solver
        p = s._dev(prim0)
        if tuple(p.shape) != s._shape():
            raise ValueError(f"primitive shape {tuple(p.shape)} != {s._shape()}")
        out = self.torch.empty(s._shape(), dtype=self.torch.float64, device=s.device)
        hz_adjoint_forward(self.adj, p.data_ptr(), out.data_ptr())
        self._keep_in = p
        self.generation += 1
        return out

    def backward(self, gprim, gcons=None):
        s = self.solver
        g = s._dev(gprim)
        gc = s._dev(gcons) if gcons is not None else None
        out = self.torch.empty(s._shape(), dtype=self.torch.float64, device=s.device)
        hz_adjoint_backward(self.adj, g.data_ptr(), gc.data_ptr() if gc is not None else None,
                            out.data_ptr())
        self._keep_g = (g, gc)
        return out

    def evolve(self, prim0):
        return _evolve_function().apply(prim0, self)


_EVOLVE_FN = None


def _evolve_function():
    """torch.autograd.Function over Adjoint.forward / Adjoint.backward (built on first use so
    that importing this module does not import torch)."""
    global _EVOLVE_FN
    if _EVOLVE_FN is None:
        import torch

        class HorizonEvolve(torch.autograd.Function):
            @staticmethod
            def forward(ctx, prim0, adj):
                out = adj.forward(prim0.detach())
                ctx.adj = adj
                ctx.generation = adj.generation
                return out

            @staticmethod
            def backward(ctx, gout):
                if ctx.adj.generation != ctx.generation:
                    raise RuntimeError("the checkpoints of this forward pass were overwritten by a "
                                       "later forward pass of the same Adjoint")
                return ctx.adj.backward(gout.contiguous()), None

        _EVOLVE_FN = HorizonEvolve
    return _EVOLVE_FN
