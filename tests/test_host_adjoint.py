"""The hand-written reverses of the adjoint path (hzn_adjoint.cuh: state algebra, conserved vector,
flux vector, wave speeds), built for the host and compared with central finite differences of the
oracle's forward pointwise functions: the vector-Jacobian product (dX/dP)^T v for random
cotangents v, in random general 3+1 metrics and in their diagonal, zero-shift reductions (the
reverse kernels' DIAG specialisation), with and without divergence cleaning.  CPU only: the same
device templates, no GPU.  The forward functions differentiated are the oracle's, so a dropped
term or a wrong sign in a reverse fails here, independently of the GPU adjoint tests (which
check the whole reverse sweep against finite differences of the forward solver)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_1102_5202_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1102_5202_gb300", "csrc")
N = 120
GAMMA = 5.0 / 3.0
CH = 0.6
TOL = 1e-6  # of the row's largest entry; measured <= 3e-8


@pytest.fixture(scope="module")
def dev():
    out = os.path.join(tempfile.mkdtemp(prefix="adj_host_"), "adjoint_host.so")
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-I", os.path.join(HERE, "host_build"), "-I", CSRC,
           os.path.join(HERE, "host_build", "adjoint_host.cpp"), "-o", out]
    subprocess.run(cmd, check=True)
    L = ctypes.CDLL(out)
    dp, ci = ctypes.POINTER(ctypes.c_double), ctypes.c_int
    L.dev_vjp.argtypes = [ctypes.c_long, ctypes.c_double, ctypes.c_double, ci, ci, ci, ci, dp, dp, dp, dp]
    L.dev_vjp.restype = None
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@pytest.fixture(scope="module", params=[0, 1], ids=["general", "diag"])
def states(request):
    """(diag, met, prim, v): moderate states (W <= 5, b^2/rho <= 10) so that the finite
    differences stay well conditioned, and standard-normal cotangents."""
    diag = request.param
    met = W.random_metric_points(N, seed=81)
    if diag:
        met[:, 1:4] = 0.0
        met[:, [5, 6, 8]] = 0.0
    met = np.ascontiguousarray(met)
    prim = np.ascontiguousarray(W.random_prim_points(N, seed=82, met=met, wmax=5.0, sigma_max=10.0))
    prim[:, 8] = np.random.Generator(np.random.PCG64(83)).uniform(-0.05, 0.05, N)
    v = np.ascontiguousarray(np.random.Generator(np.random.PCG64(84)).standard_normal((N, 9)))
    return diag, met, prim, v


def _fd_vjp(fwd, prim, v, nfield):
    """sum_k v_k dX_k/dP_j by the five-point central difference (fourth order) along each
    primitive, differenced componentwise before the weighting.  Step 1e-3 of the value; density
    and pressure (down to 1e-9 here, the scale the speeds vary on) take purely relative steps,
    the other fields a floor of 1e-3."""
    g = np.zeros((prim.shape[0], nfield))
    for k in range(nfield):
        h = 1e-3 * np.maximum(np.abs(prim[:, k]), 0.0 if k < 2 else 1e-3)
        f = []
        for m in (-2.0, -1.0, 1.0, 2.0):
            q = prim.copy()
            q[:, k] += m * h
            f.append(fwd(q))
        g[:, k] = ((f[0] - f[3] + 8.0 * (f[2] - f[1])) * v).sum(axis=1) / (12.0 * h)
    return g


def _rel(a, b):
    scale = np.maximum(np.abs(b).max(axis=1, keepdims=True), 1e-300)
    return float((np.abs(a - b) / scale).max())


def _run(dev, clean, diag, what, d, met, prim, v):
    out = np.zeros((N, 9))
    dev.dev_vjp(N, GAMMA, CH, clean, diag, what, d, _p(met), _p(prim), _p(v), _p(out))
    return out


@pytest.mark.parametrize("clean", [0, 1])
def test_conserved_vector_reverse_matches_finite_differences(dev, states, clean):
    diag, met, prim, v = states
    nf = 9 if clean else 8
    vv = v.copy()
    vv[:, nf:] = 0.0
    got = _run(dev, clean, diag, 0, 0, met, prim, vv)
    opts = O.make_opts(GAMMA, cleaning=bool(clean))
    want = _fd_vjp(lambda p: O.prim2cons(opts, met, p), prim, vv, nf)
    assert _rel(got[:, :nf], want) < TOL
    if not clean:
        assert np.all(got[:, 8] == 0.0)


@pytest.mark.parametrize("clean", [0, 1])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_flux_vector_reverse_matches_finite_differences(dev, states, clean, d):
    diag, met, prim, v = states
    nf = 9 if clean else 8
    vv = v.copy()
    vv[:, nf:] = 0.0
    got = _run(dev, clean, diag, 1, d, met, prim, vv)
    opts = O.make_opts(GAMMA, cleaning=bool(clean), ch=CH)
    want = _fd_vjp(lambda p: O.flux(opts, d, met, p), prim, vv, nf)
    assert _rel(got[:, :nf], want) < TOL


@pytest.mark.parametrize("d", [0, 1, 2])
def test_wave_speed_reverse_matches_finite_differences(dev, states, d):
    """Weights on (lambda-, lambda+); the speeds do not depend on psi."""
    diag, met, prim, v = states
    w2 = np.ascontiguousarray(v[:, :2])
    vv = np.zeros((N, 9))
    vv[:, :2] = w2
    got = _run(dev, 0, diag, 2, d, met, prim, vv)
    opts = O.make_opts(GAMMA)
    want = _fd_vjp(lambda p: O.speeds(opts, d, met, p), prim, w2, 8)
    assert _rel(got[:, :8], want) < TOL
