"""Op-counting run of the oracle (``opcount.cpp``): the floating-point operations of one RK3
step of the oracle's method, per phase and per kind.

TEST AND MEASUREMENT INFRASTRUCTURE, NOT PRODUCT CODE (same rules as the rest of ``oracle/``).
The counts define the algorithmic flops per zone update that the FP64 path's ALU roofline uses;
``write_counts.py`` beside this file stores them for the benchmark workload.

Counting conventions (stated in full in ``opcount.cpp``): +, -, *, / and sqrt one flop each;
operations with a structural zero operand (literal zeros, vanishing metric components) free;
metric-only work in the ``geometry`` bucket (computed once for a static spacetime); the
recovery's double-precision root solve added per call from its iteration count.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import Grid, Opts, _dp, _f64

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "opcount.cpp")
_DEP = os.path.join(_HERE, "hz_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libhzopcount.so")
_lock = threading.Lock()
_lib = None

PHASES = ("geometry", "recon", "face_state", "flux", "speeds", "hlle", "divergence", "sources",
          "update", "c2p", "cfl")
OPS = ("add", "mul", "div", "sqrt")


def build(force: bool = False) -> str:
    """Compile the counting library (g++, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_DEP))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            L.hzo_opcount_step.argtypes = [P(Grid), P(Opts), P(ctypes.c_double), P(ctypes.c_double),
                                           ctypes.c_double, ctypes.c_int, P(ctypes.c_longlong),
                                           P(ctypes.c_longlong), P(ctypes.c_longlong), P(ctypes.c_double),
                                           P(ctypes.c_long), P(ctypes.c_long)]
            L.hzo_opcount_step.restype = None
            L.hzo_opcount_max_unit.restype = ctypes.c_long
            assert L.hzo_opcount_nphase() == len(PHASES) and L.hzo_opcount_nop() == len(OPS)
            _lib = L
    return _lib


def count_step(grid: Grid, opts: Opts, met, prim, dt: float, check_rhs: bool = True) -> dict:
    """Counts of one RK3 step of size dt from the primitive state ``prim`` (9, nz, ny, nx).

    Returns ``tally`` (phases x ops, int64: the distinct operations each face's and each cell's
    results and decisions depend on, the algorithmic count), ``raw`` (every operation the
    oracle executes), ``per_zu`` / ``raw_per_zu`` (phase -> flops per zone update: the step's
    counts over the cell count), ``check`` (with ``check_rhs``: raw count of the phased
    right-hand side minus the oracle rhs()'s, per stage: zeros), ``vdiff`` (largest difference of
    their values),
    ``iters`` and ``calls`` of the recovery's root solve."""
    met, prim = _f64(met), _f64(prim)
    raw = np.zeros((len(PHASES), len(OPS)), dtype=np.int64)
    tally = np.zeros((len(PHASES), len(OPS)), dtype=np.int64)
    check = np.zeros(3, dtype=np.int64)
    vdiff = ctypes.c_double(0.0)
    iters, calls = ctypes.c_long(0), ctypes.c_long(0)
    llp = ctypes.POINTER(ctypes.c_longlong)
    lib().hzo_opcount_step(ctypes.byref(grid), ctypes.byref(opts), _dp(met), _dp(prim), float(dt),
                           int(bool(check_rhs)), raw.ctypes.data_as(llp), tally.ctypes.data_as(llp), check.ctypes.data_as(llp),
                           ctypes.byref(vdiff), ctypes.byref(iters), ctypes.byref(calls))
    ncell = int(grid.n[0] * grid.n[1] * grid.n[2])
    per_zu = {ph: float(tally[p].sum()) / ncell for p, ph in enumerate(PHASES)}
    raw_per_zu = {ph: float(raw[p].sum()) / ncell for p, ph in enumerate(PHASES)}
    return dict(tally=tally, raw=raw, per_zu=per_zu, raw_per_zu=raw_per_zu, check=check,
                vdiff=vdiff.value, iters=iters.value, calls=calls.value, ncell=ncell)


def step_flops_per_zu(result: dict) -> float:
    """Algorithmic flops per zone update of a count: every phase but the static geometry."""
    return sum(v for k, v in result["per_zu"].items() if k != "geometry")
