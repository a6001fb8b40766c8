"""The CUDA path's pointwise physics (hzn_physics.cuh: metric geometry, state algebra, conserved
and flux vectors, wave speeds in both the plain and the FP64 kernel's scaled form, and the
recovery) built for the host and compared with the oracle's pointwise functions on random
states of high Lorentz factor and magnetisation, in random general 3+1 metrics and in their
diagonal, zero-shift reductions through the kernels' DIAG specialisation.  CPU only: the
same device templates, no GPU."""
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
N = 400
GAMMA = 5.0 / 3.0
CH = 0.6


@pytest.fixture(scope="module")
def dev():
    out = os.path.join(tempfile.mkdtemp(prefix="phys_host_"), "physics_host.so")
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-I", os.path.join(HERE, "host_build"), "-I", CSRC,
           os.path.join(HERE, "host_build", "physics_host.cpp"), "-o", out]
    subprocess.run(cmd, check=True)
    L = ctypes.CDLL(out)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    ci = ctypes.c_int
    L.dev_prim2cons.argtypes = [ctypes.c_long, ctypes.c_double, ci, ci, dp, dp, dp]
    L.dev_flux.argtypes = [ctypes.c_long, ctypes.c_double, ctypes.c_double, ci, ci, ci, dp, dp, dp]
    L.dev_speeds.argtypes = [ctypes.c_long, ctypes.c_double, ci, ci, dp, dp, dp, dp]
    L.dev_con2prim.argtypes = [ctypes.c_long, ctypes.c_double, ci, ci, dp, dp, dp,
                               ctypes.c_double, ci, dp, ip]
    L.dev_reconstruct.argtypes = [ci, ctypes.c_long, dp, dp, dp]
    L.dev_source.argtypes = [ctypes.c_long, ctypes.c_double, ci, dp, dp, dp, dp]
    for f in (L.dev_prim2cons, L.dev_flux, L.dev_speeds, L.dev_con2prim, L.dev_reconstruct, L.dev_source):
        f.restype = None
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@pytest.fixture(scope="module", params=[0, 1], ids=["general", "diag"])
def states(request):
    """(diag, met, prim): general 3+1 metrics, or the same with zero shift and diagonal gamma
    (the kernels' DIAG specialisation)."""
    diag = request.param
    met = W.random_metric_points(N, seed=71)
    if diag:
        met[:, 1:4] = 0.0
        met[:, [5, 6, 8]] = 0.0
    met = np.ascontiguousarray(met)
    prim = np.ascontiguousarray(W.random_prim_points(N, seed=72, met=met, wmax=10.0, sigma_max=100.0))
    prim[:, 8] = np.random.Generator(np.random.PCG64(73)).uniform(-0.05, 0.05, N)
    return diag, met, prim


def _rel(a, b):
    """Largest componentwise error over the state's own scale (the row's largest magnitude)."""
    scale = np.maximum(np.abs(b).max(axis=1, keepdims=True), 1e-300)
    return float((np.abs(a - b) / scale).max())


@pytest.mark.parametrize("clean", [0, 1])
def test_conserved_vector_matches_oracle(dev, states, clean):
    diag, met, prim = states
    got = np.zeros((N, 9))
    dev.dev_prim2cons(N, GAMMA, clean, diag, _p(met), _p(prim), _p(got))
    want = O.prim2cons(O.make_opts(GAMMA, cleaning=bool(clean)), met, prim)
    cols = slice(0, 9 if clean else 8)
    assert _rel(got[:, cols], want[:, cols]) < 5e-12


@pytest.mark.parametrize("clean", [0, 1])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_flux_vector_matches_oracle(dev, states, clean, d):
    diag, met, prim = states
    got = np.zeros((N, 9))
    dev.dev_flux(N, GAMMA, CH, clean, diag, d, _p(met), _p(prim), _p(got))
    want = O.flux(O.make_opts(GAMMA, cleaning=bool(clean), ch=CH), d, met, prim)
    cols = slice(0, 9 if clean else 8)
    assert _rel(got[:, cols], want[:, cols]) < 5e-12  # measured <= 9e-13 (W <= 10, b^2/rho <= 100)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_wave_speeds_both_forms_match_oracle(dev, states, d):
    """The plain quadratic (mixed and pair paths) and the FP64 kernel's form (multiplied through
    by w(w + b^2), halved linear coefficient) give the oracle's speeds."""
    diag, met, prim = states
    lam = np.zeros((N, 2))
    lam_q = np.zeros((N, 2))
    dev.dev_speeds(N, GAMMA, diag, d, _p(met), _p(prim), _p(lam), _p(lam_q))
    want = O.speeds(O.make_opts(GAMMA), d, met, prim)
    assert np.abs(lam - want).max() < 1e-12
    assert np.abs(lam_q - want).max() < 1e-12
    assert np.all(lam[:, 0] <= lam[:, 1])


def test_recovery_returns_the_state_and_matches_oracle(dev, states):
    """From the conserved vector of each state and a guess 10 % off, the device recovery returns
    the state (round trip) and the oracle's root."""
    diag, met, prim = states
    cons = O.prim2cons(O.make_opts(GAMMA, cleaning=True), met, prim)
    guess = prim.copy()
    guess[:, 0] *= 1.1
    guess[:, 1] *= 0.9
    guess[:, 2:5] *= 0.95
    got = np.zeros((N, 9))
    status = np.zeros(N, dtype=np.int32)
    dev.dev_con2prim(N, GAMMA, 1, diag, _p(met), _p(cons), _p(guess), 1e-12, 50, _p(got),
                     status.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    assert np.all(status == 0)
    assert _rel(got, prim) < 1e-11  # measured 2.7e-13
    orc, _, _ = O.cons2prim(O.make_opts(GAMMA, cleaning=True), met, cons, guess)
    assert _rel(got, orc) < 1e-11


def test_metric_source_matches_oracle(dev, states):
    """The kernels' source algebra (T^{ab} of tup_of contracted with metric differences by tdg)
    against the oracle's 1/2 sqrt(-g) T^{ab} d_i g_ab, for random symmetric derivatives (diagonal
    ones for the DIAG specialisation, whose metrics keep zero shift and diagonal gamma)."""
    diag, met, prim = states
    rng = np.random.Generator(np.random.PCG64(75))
    dg = rng.uniform(-0.3, 0.3, (N, 3, 4, 4))
    dg = 0.5 * (dg + dg.transpose(0, 1, 3, 2))
    if diag:
        dg = dg * np.eye(4)[None, None]
    dg = np.ascontiguousarray(dg.reshape(N, 48))
    got = np.zeros((N, 4))
    dev.dev_source(N, GAMMA, diag, _p(met), _p(dg), _p(prim), _p(got))
    want = O.source_pointwise(O.make_opts(GAMMA), met, dg, prim)
    assert _rel(got, want) < 1e-12


def _profiles():
    """1-D arrays with smooth parts, jumps, plateaus (exact zero differences), isolated extrema
    and values spanning many decades."""
    rng = np.random.Generator(np.random.PCG64(74))
    x = np.linspace(0.0, 1.0, 400)
    out = [np.sin(7 * x) + 0.3 * np.cos(31 * x),
           np.where(x < 0.4, 1.0, 0.125) + np.where(x > 0.7, 2.0, 0.0),
           np.round(rng.uniform(0, 4, 400)) * 0.25,
           10.0 ** rng.uniform(-12, 2, 400),
           np.exp(-((x - 0.5) / 0.05) ** 2)]
    return [np.ascontiguousarray(q) for q in out]


def test_mc_reconstruction_is_the_oracles_bit_for_bit(dev):
    """The FP64 MC faces (bit-pattern minimum, exponent-arithmetic quarter) are the numbers of
    the oracle's floating-point MC, exactly."""
    for q in _profiles():
        n = len(q)
        left, right = np.full(n, np.nan), np.full(n, np.nan)
        dev.dev_reconstruct(0, n, _p(q), _p(left), _p(right))
        wl, wr = O.reconstruct_1d(O.RECON_MC, q)
        assert np.array_equal(left[3:n - 2], wl[3:n - 2]) and np.array_equal(right[3:n - 2], wr[3:n - 2])


def test_ppm_and_pair_mc_reconstruction_match_oracle(dev):
    for q in _profiles():
        n = len(q)
        scale = np.abs(q).max()
        left, right = np.full(n, np.nan), np.full(n, np.nan)
        dev.dev_reconstruct(1, n, _p(q), _p(left), _p(right))
        wl, wr = O.reconstruct_1d(O.RECON_PPM, q)
        s = slice(3, n - 2)
        assert np.abs(left[s] - wl[s]).max() <= 1e-14 * scale and np.abs(right[s] - wr[s]).max() <= 1e-14 * scale
        dev.dev_reconstruct(2, n, _p(q), _p(left), _p(right))
        wl, wr = O.reconstruct_1d(O.RECON_MC, q)
        assert np.abs(left[s] - wl[s]).max() <= 1e-13 * scale and np.abs(right[s] - wr[s]).max() <= 1e-13 * scale
