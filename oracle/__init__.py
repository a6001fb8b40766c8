"""FP64 CPU oracle of the HORIZON GRMHD finite-volume update (arXiv:1102.5202).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  It shares nothing with the CUDA path
except the seeded inputs of ``paper_1102_5202_gb300.workloads``.

The arithmetic lives in ``hz_oracle.cpp`` (plain C++, FP64, compiled with
``-ffp-contract=off``); this module builds it with g++ and marshals numpy arrays.

Array conventions (all float64, C-contiguous):
  * grid primitives / conserved: shape (9, nz, ny, nx); metric: (10, nz+2gz, ny+2gy, nx+2gx)
    with one ghost layer on every axis with more than one cell;
  * pointwise helpers take (n, 10) metric rows and (n, 9) primitive / conserved rows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hz_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhzoracle.so")
_lock = threading.Lock()
_lib = None


class Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("bc", ctypes.c_int * 3), ("dx", ctypes.c_double * 3)]


class Opts(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double),
        ("cleaning", ctypes.c_int),
        ("ch", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("rho_floor", ctypes.c_double),
        ("p_floor", ctypes.c_double),
        ("atm_K", ctypes.c_double),
        ("c2p_maxit", ctypes.c_int),
        ("rho_atm", ctypes.c_double),
        ("recon", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            dp = P(ctypes.c_double)
            ip = P(ctypes.c_int)
            gp, op = P(Grid), P(Opts)
            L.hzo_prim2cons.argtypes = [ctypes.c_long, op, dp, dp, dp]
            L.hzo_cons2prim.argtypes = [ctypes.c_long, op, dp, dp, dp, dp, ip, ip]
            L.hzo_cons2prim.restype = ctypes.c_long
            L.hzo_recover.argtypes = [ctypes.c_long, op, dp, dp, dp, dp, ip]
            L.hzo_recover.restype = ctypes.c_long
            L.hzo_flux.argtypes = [ctypes.c_long, op, ctypes.c_int, dp, dp, dp]
            L.hzo_speeds.argtypes = [ctypes.c_long, op, ctypes.c_int, dp, dp, dp]
            L.hzo_state.argtypes = [ctypes.c_long, op, dp, dp, dp]
            L.hzo_source_pointwise.argtypes = [ctypes.c_long, op, dp, dp, dp, dp]
            L.hzo_tensors.argtypes = [ctypes.c_long, op, dp, dp, dp, dp, dp]
            L.hzo_grid_prim2cons.argtypes = [gp, op, dp, dp, dp]
            L.hzo_rhs.argtypes = [gp, op, dp, dp, dp]
            L.hzo_rhs_source.argtypes = [gp, op, dp, dp, dp]
            L.hzo_max_speed.argtypes = [gp, op, dp, dp]
            L.hzo_max_speed.restype = ctypes.c_double
            L.hzo_step.argtypes = [gp, op, dp, dp, dp, ctypes.c_double]
            L.hzo_step.restype = ctypes.c_long
            L.hzo_evolve.argtypes = [gp, op, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_long, dp, P(ctypes.c_long)]
            L.hzo_evolve.restype = ctypes.c_long
            L.hzo_evolve_cs.argtypes = [gp, op, dp, dp, dp, ctypes.c_double, ctypes.c_long, dp, dp, dp,
                                        dp]
            L.hzo_evolve_cs.restype = ctypes.c_long
            L.hzo_reconstruct_1d.argtypes = [ctypes.c_int, ctypes.c_long, dp, dp, dp]
            L.hzo_num_threads.restype = ctypes.c_int
            L.hzo_set_num_threads.argtypes = [ctypes.c_int]
            L.hzo_set_num_threads.restype = None
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


RECON_MC, RECON_PPM = 0, 1


def make_opts(gamma: float, cleaning: bool = False, ch: float = 0.0, kappa: float = 0.0,
              rho_floor: float = 1e-12, p_floor: float = 1e-14, atm_K: float = 0.0,
              c2p_maxit: int = 200, rho_atm: float = 0.0, recon: int = RECON_MC) -> Opts:
    return Opts(float(gamma), int(bool(cleaning)), float(ch), float(kappa), float(rho_floor),
                float(p_floor), float(atm_K), int(c2p_maxit), float(rho_atm), int(recon))


def make_grid(n, dx, bc) -> Grid:
    g = Grid()
    for d in range(3):
        g.n[d] = int(n[d])
        g.dx[d] = float(dx[d])
        g.bc[d] = int(bc[d])
    return g


def num_threads() -> int:
    return int(lib().hzo_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the grid operations from now on."""
    lib().hzo_set_num_threads(int(n))


# ---------------------------------------------------------------- pointwise helpers
def prim2cons(opts: Opts, met, prim) -> np.ndarray:
    met, prim = _f64(met), _f64(prim)
    n = prim.shape[0]
    out = np.empty((n, 9))
    lib().hzo_prim2cons(n, ctypes.byref(opts), _dp(met), _dp(prim), _dp(out))
    return out


def cons2prim(opts: Opts, met, cons, guess=None):
    """Returns (prim, status, iters); status 1 marks a failed recovery."""
    met, cons = _f64(met), _f64(cons)
    n = cons.shape[0]
    out = np.zeros((n, 9))
    st = np.zeros(n, dtype=np.int32)
    it = np.zeros(n, dtype=np.int32)
    g = None
    if guess is not None:
        guess = _f64(guess)
        g = _dp(guess)
    lib().hzo_cons2prim(n, ctypes.byref(opts), _dp(met), _dp(cons), g, _dp(out),
                        st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                        it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out, st, it


def recover(opts: Opts, met, cons, guess=None):
    """Recovery with the step's atmosphere and floor rules.
    Returns (prim, cons_after, status)."""
    met = _f64(met)
    cons = _f64(cons).copy()
    n = cons.shape[0]
    out = np.zeros((n, 9))
    st = np.zeros(n, dtype=np.int32)
    g = None
    if guess is not None:
        guess = _f64(guess)
        g = _dp(guess)
    lib().hzo_recover(n, ctypes.byref(opts), _dp(met), _dp(cons), g, _dp(out),
                      st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out, cons, st


def flux(opts: Opts, d: int, met, prim) -> np.ndarray:
    met, prim = _f64(met), _f64(prim)
    out = np.empty((prim.shape[0], 9))
    lib().hzo_flux(prim.shape[0], ctypes.byref(opts), d, _dp(met), _dp(prim), _dp(out))
    return out


def speeds(opts: Opts, d: int, met, prim) -> np.ndarray:
    met, prim = _f64(met), _f64(prim)
    out = np.empty((prim.shape[0], 2))
    lib().hzo_speeds(prim.shape[0], ctypes.byref(opts), d, _dp(met), _dp(prim), _dp(out))
    return out


def state(opts: Opts, met, prim) -> np.ndarray:
    """(n, 14): u^mu, b^mu, b^2, W, sqrt(gamma), alpha, T^t_t, w."""
    met, prim = _f64(met), _f64(prim)
    out = np.empty((prim.shape[0], 14))
    lib().hzo_state(prim.shape[0], ctypes.byref(opts), _dp(met), _dp(prim), _dp(out))
    return out


def source_pointwise(opts: Opts, met, dg, prim) -> np.ndarray:
    met, dg, prim = _f64(met), _f64(dg), _f64(prim)
    out = np.empty((prim.shape[0], 4))
    lib().hzo_source_pointwise(prim.shape[0], ctypes.byref(opts), _dp(met), _dp(dg), _dp(prim),
                               _dp(out))
    return out


def tensors(opts: Opts, met, prim):
    met, prim = _f64(met), _f64(prim)
    n = prim.shape[0]
    T, g, gi = np.empty((n, 4, 4)), np.empty((n, 4, 4)), np.empty((n, 4, 4))
    lib().hzo_tensors(n, ctypes.byref(opts), _dp(met), _dp(prim), _dp(T), _dp(g), _dp(gi))
    return T, g, gi


# ---------------------------------------------------------------- grid operations
def grid_prim2cons(grid: Grid, opts: Opts, met, prim) -> np.ndarray:
    met, prim = _f64(met), _f64(prim)
    out = np.empty_like(prim)
    lib().hzo_grid_prim2cons(ctypes.byref(grid), ctypes.byref(opts), _dp(met), _dp(prim), _dp(out))
    return out


def rhs(grid: Grid, opts: Opts, met, prim) -> np.ndarray:
    met, prim = _f64(met), _f64(prim)
    out = np.empty_like(prim)
    lib().hzo_rhs(ctypes.byref(grid), ctypes.byref(opts), _dp(met), _dp(prim), _dp(out))
    return out


def rhs_source(grid: Grid, opts: Opts, met, prim) -> np.ndarray:
    """The metric source and cleaning damping of ``rhs`` alone (no flux difference)."""
    met, prim = _f64(met), _f64(prim)
    out = np.empty_like(prim)
    lib().hzo_rhs_source(ctypes.byref(grid), ctypes.byref(opts), _dp(met), _dp(prim), _dp(out))
    return out


def max_speed(grid: Grid, opts: Opts, met, prim) -> float:
    met, prim = _f64(met), _f64(prim)
    return float(lib().hzo_max_speed(ctypes.byref(grid), ctypes.byref(opts), _dp(met), _dp(prim)))


def step(grid: Grid, opts: Opts, met, prim, cons, dt: float):
    """One RK3 step; returns (prim, cons, failures) as new arrays."""
    met = _f64(met)
    prim = _f64(prim).copy()
    cons = _f64(cons).copy()
    nf = lib().hzo_step(ctypes.byref(grid), ctypes.byref(opts), _dp(met), _dp(prim), _dp(cons),
                        float(dt))
    return prim, cons, int(nf)


def evolve(grid: Grid, opts: Opts, met, prim, cons, t_end: float, cfl: float,
           fixed_dt: float = 0.0, max_steps: int = 1 << 40):
    """Evolve to t_end; returns (prim, cons, steps, t, failures)."""
    met = _f64(met)
    prim = _f64(prim).copy()
    cons = _f64(cons).copy()
    t = ctypes.c_double(0.0)
    nf = ctypes.c_long(0)
    steps = lib().hzo_evolve(ctypes.byref(grid), ctypes.byref(opts), _dp(met), _dp(prim), _dp(cons),
                             float(t_end), float(cfl), float(fixed_dt), int(max_steps),
                             ctypes.byref(t), ctypes.byref(nf))
    return prim, cons, int(steps), float(t.value), int(nf.value)


def evolve_cs(grid: Grid, opts: Opts, met, prim, dprim, h: float, dt: float, nsteps: int):
    """Complex-step directional derivative of the state after nsteps fixed steps of size dt.

    Runs the scheme on prim + i h dprim and returns (prim_end, dprim_end, cons_end, dcons_end,
    failures) with dX_end = Im(X_end(prim + i h dprim)) / h: the derivative of the discrete map
    (branch decisions frozen at the real state) up to O(h^2) and round-off, since no difference
    of nearby values is formed."""
    met = _f64(met)
    pre = _f64(prim)
    pim = _f64(dprim) * float(h)
    ore, oim = np.empty_like(pre), np.empty_like(pre)
    cre, cim = np.empty_like(pre), np.empty_like(pre)
    nf = lib().hzo_evolve_cs(ctypes.byref(grid), ctypes.byref(opts), _dp(met), _dp(pre), _dp(pim),
                             float(dt), int(nsteps), _dp(ore), _dp(oim), _dp(cre), _dp(cim))
    return ore, oim / float(h), cre, cim / float(h), int(nf)


def reconstruct_1d(recon: int, q):
    """(left, right) face states of a 1-D array at the faces between cells c-1 and c, for
    c = 3 .. n-3 (entries outside that range are NaN)."""
    q = _f64(q)
    n = q.shape[0]
    left, right = np.full(n, np.nan), np.full(n, np.nan)
    lib().hzo_reconstruct_1d(int(recon), n, _dp(q), _dp(left), _dp(right))
    return left, right
