"""The substep kernel's spatial operator L(P) (§2.2: reconstruction, HLLE face fluxes with the
lapse / shift / sqrt(gamma) weights, flux divergence, metric source, cleaning damping), built
for the host from the product's face templates (`face_flux` in FP64 with MC or PPM,
`face_flux_dw` with its cyclic rotation of the axes, the mixed path's FP32 faces) and the DIAG
geometry tables, and compared with the oracle's `rhs` field by field on small grids: a curved
diagonal-metric star, smooth periodic data in a general metric (shift, non-diagonal gamma) in
2-D and 3-D with a non-zero cleaning scalar, and a discontinuous shock tube along each axis.
CPU only: the same device templates, no GPU.  The harness pads the arrays with NaN and uses odd
pitches, so a read outside the stencil or a wrong stride fails here.  Also from the same header:
the recovery with the atmosphere and floor rules (`recover`) against the oracle's recovery of the
step, and the CFL rate (`cell_max_speed`: the largest per-cell sum over axes of |lambda| / dx)
against the oracle's."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
import parity
from paper_1102_5202_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1102_5202_gb300", "csrc")

# largest error of a field over that field's largest magnitude; measured: FP64 <= 3.1e-14,
# double-word faces <= 1.3e-13, mixed FP32 faces <= 2.0e-6
TOL = {"fp64": 1e-12, "dw": 1e-11, "mixed": 1e-5}
PAIR = {"fp64": 0, "dw": 1, "mixed": 2}


@pytest.fixture(scope="module")
def dev():
    out = os.path.join(tempfile.mkdtemp(prefix="rhs_host_"), "rhs_host.so")
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-I", os.path.join(HERE, "host_build"), "-I", CSRC,
           os.path.join(HERE, "host_build", "rhs_host.cpp"), "-o", out]
    subprocess.run(cmd, check=True)
    L = ctypes.CDLL(out)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    ci, cd = ctypes.c_int, ctypes.c_double
    L.dev_rhs.argtypes = [ip, dp, ip, cd, ci, cd, cd, ci, ci, ci, dp, dp, dp]
    L.dev_rhs.restype = ci
    L.dev_recover.argtypes = [ctypes.c_long, cd, ci, ci, cd, cd, cd, cd, ci, cd, ci, dp, dp, dp, dp, ip]
    L.dev_recover.restype = None
    L.dev_max_speed.argtypes = [ip, dp, ip, cd, ci, cd, ci, dp, dp]
    L.dev_max_speed.restype = cd
    L.dev_rest_max_speed.argtypes = [ip, dp, ip, cd, ci, cd, dp, dp]
    L.dev_rest_max_speed.restype = cd
    return L


def _general(n, seed):
    P = W.with_periodic_metric(W.smooth_periodic(n, seed=seed), parity.general_metric)
    P.cleaning, P.ch, P.kappa = True, 0.6, 0.3
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    P.prim[8] = 0.02 * rng.uniform(-1.0, 1.0, P.prim[8].shape)
    return P


def _cases():
    blob = W.blob3d(12)
    tube = W.balsara1(40)
    tube.cleaning, tube.ch, tube.kappa = True, 0.7, 0.2
    return {
        "blob12_diag": (blob, 1),
        "blob12_general_code": (blob, 0),
        "smooth_general_3d": (_general((10, 8, 6), 5), 0),
        "smooth_general_2d": (_general((12, 9, 1), 6), 0),
        "balsara1_x": (tube, 1),
        "balsara1_y": (parity.tile_tube(tube, 1), 1),
        "balsara1_z": (parity.tile_tube(tube, 2), 0),
    }


CASES = _cases()


def _rhs(dev, P, diag, recon, path, clean):
    n = (ctypes.c_int * 3)(*P.n)
    dx = (ctypes.c_double * 3)(*P.dx)
    bc = (ctypes.c_int * 3)(*P.bc)
    met = np.ascontiguousarray(P.metric, dtype=np.float64)
    prim = np.ascontiguousarray(P.prim, dtype=np.float64)
    got = np.zeros_like(prim)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = dev.dev_rhs(n, dx, bc, P.gamma, int(clean), P.ch, P.kappa, diag, recon, PAIR[path],
                     met.ctypes.data_as(dp), prim.ctypes.data_as(dp), got.ctypes.data_as(dp))
    assert rc == 0
    opts = O.make_opts(P.gamma, cleaning=bool(clean), ch=P.ch, kappa=P.kappa, recon=recon)
    want = O.rhs(O.make_grid(P.n, P.dx, P.bc), opts, met, prim)
    return got, want


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("path,recon", [("fp64", 0), ("fp64", 1), ("dw", 0), ("mixed", 0), ("mixed", 1)])
@pytest.mark.parametrize("clean", [0, 1])
def test_spatial_operator_matches_oracle(dev, case, path, recon, clean):
    P, diag = CASES[case]
    got, want = _rhs(dev, P, diag, recon, path, clean)
    nf = 9 if clean else 8
    assert np.all(np.isfinite(got[:nf]))
    for f in range(nf):
        scale = np.abs(want[f]).max()
        if scale == 0.0:
            assert np.all(got[f] == 0.0), f
            continue
        err = np.abs(got[f] - want[f]).max() / scale
        assert err < TOL[path], (case, path, recon, f, err)
    if not clean:
        assert np.all(got[8] == 0.0)


def test_cases_exercise_the_method():
    """The cases are not trivial: every active axis carries flux differences, the star and the
    general metric give metric sources, and the cleaning scalar is non-zero."""
    P, _ = CASES["smooth_general_3d"]
    assert np.abs(P.prim[8]).max() > 0.01
    assert np.abs(P.metric[1:4]).max() > 0.01 and np.abs(P.metric[[5, 6, 8]]).max() > 0.005
    P, _ = CASES["blob12_diag"]
    assert np.all(P.metric[1:4] == 0.0) and np.all(P.metric[[5, 6, 8]] == 0.0)
    assert np.ptp(P.metric[0]) > 0.01
    P, _ = CASES["balsara1_x"]
    assert np.ptp(P.prim[0]) > 0.5


def _bad_energy(cons):
    cons[::7, 1] = -0.3 * cons[::7, 0]  # energy below the rest mass: no physical state


@pytest.mark.parametrize("diag", [0, 1])
@pytest.mark.parametrize("clean", [0, 1])
@pytest.mark.parametrize("rule", ["plain", "atmosphere", "pressure_floor", "unphysical"])
@pytest.mark.parametrize("one_d", [0, 1], ids=["newton2d", "newton1d"])
def test_recovery_with_atmosphere_and_floors_matches_oracle(dev, diag, clean, rule, one_d):
    """Same failures, same resets, same primitive and rewritten conserved states, with either
    of the kernels' Newton schemes (§3.2 names a one- and a two-dimensional recovery)."""
    n, gamma = 400, 5.0 / 3.0
    rho_floor, p_floor, atm_K, rho_atm, mutate = 1e-12, 1e-14, 0.0, 0.0, None
    if rule == "atmosphere":
        rho_floor, atm_K, rho_atm = 1e-7, 100.0, 1e-5
    elif rule == "pressure_floor":
        p_floor = 1e-4
    elif rule == "unphysical":
        mutate = _bad_energy
    met = W.random_metric_points(n, seed=91)
    if diag:
        met[:, 1:4] = 0.0
        met[:, [5, 6, 8]] = 0.0
    met = np.ascontiguousarray(met)
    prim = np.ascontiguousarray(W.random_prim_points(n, seed=92, met=met, wmax=5.0, sigma_max=10.0))
    prim[:, 8] = np.random.Generator(np.random.PCG64(93)).uniform(-0.05, 0.05, n) if clean else 0.0
    opts = O.make_opts(gamma, cleaning=bool(clean), rho_floor=rho_floor, p_floor=p_floor, atm_K=atm_K,
                       rho_atm=rho_atm)
    cons = O.prim2cons(opts, met, prim)
    if mutate is not None:
        mutate(cons)
    rng = np.random.Generator(np.random.PCG64(94))
    guess = np.ascontiguousarray(prim * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, prim.shape)))
    want_p, want_u, want_s = O.recover(opts, met, cons, guess)
    p_atm = max(atm_K * rho_floor ** gamma if atm_K > 0 else p_floor, p_floor)
    got_u = np.ascontiguousarray(cons.copy())
    got_p = np.zeros((n, 9))
    got_s = np.zeros(n, dtype=np.int32)
    dp = ctypes.POINTER(ctypes.c_double)
    dev.dev_recover(n, gamma, clean, diag, rho_floor, p_floor, p_atm, rho_atm, 200, 1e-14, one_d,
                    met.ctypes.data_as(dp), got_u.ctypes.data_as(dp), guess.ctypes.data_as(dp),
                    got_p.ctypes.data_as(dp), got_s.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    nf = 9 if clean else 8
    assert np.array_equal(got_s, want_s)
    if rule == "unphysical":
        assert want_s.sum() > 0
    if rule in ("atmosphere", "pressure_floor"):
        assert np.any(np.abs(want_u - cons).max(axis=1) > 0)  # some cells were reset
    for got, want in ((got_p, want_p), (got_u, want_u)):
        scale = np.maximum(np.abs(want[:, :nf]).max(axis=1, keepdims=True), 1e-300)
        assert (np.abs(got[:, :nf] - want[:, :nf]) / scale).max() < 1e-12  # measured <= 9.3e-14


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("clean", [0, 1])
def test_cfl_maximum_matches_oracle(dev, case, clean):
    P, diag = CASES[case]
    n = (ctypes.c_int * 3)(*P.n)
    dx = (ctypes.c_double * 3)(*P.dx)
    bc = (ctypes.c_int * 3)(*P.bc)
    met = np.ascontiguousarray(P.metric, dtype=np.float64)
    prim = np.ascontiguousarray(P.prim, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    got = dev.dev_max_speed(n, dx, bc, P.gamma, clean, P.ch, diag, met.ctypes.data_as(dp),
                            prim.ctypes.data_as(dp))
    want = O.max_speed(O.make_grid(P.n, P.dx, P.bc), O.make_opts(P.gamma, cleaning=bool(clean), ch=P.ch),
                       met, prim)
    assert got == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("clean", [0, 1])
def test_rest_state_cfl_rate_closed_form(dev, clean, seed):
    """The closed-form CFL rate the kernels take for cells at rest on a zero-shift diagonal
    metric (rest_cfl_rate: lambda = -+ c alpha sqrt(gamma^dd) with c^2 = (Gamma p + b^2)/(w + b^2),
    b^2 = alpha^2 gamma_ij B^i B^j, widened to the cleaning speed) against the oracle's general
    dispersion-relation roots, on the capped-Schwarzschild blob metric with random densities,
    pressures and fields spanning six decades, magnetically and thermally dominated cells both
    (the grid maximum is one cell's rate; each seed selects another cell)."""
    P = W.blob3d(12)
    rng = np.random.Generator(np.random.PCG64(17 + seed))
    shape = P.prim.shape[1:]
    prim = np.zeros_like(P.prim)
    prim[0] = 10.0 ** rng.uniform(-6, 0, shape)
    prim[1] = 10.0 ** rng.uniform(-8, 0, shape)
    prim[5:8] = rng.uniform(-1, 1, (3,) + shape) * 10.0 ** rng.uniform(-4, 0, shape)
    ch = 0.3
    n = (ctypes.c_int * 3)(*P.n)
    dx = (ctypes.c_double * 3)(*P.dx)
    bc = (ctypes.c_int * 3)(*P.bc)
    met = np.ascontiguousarray(P.metric, dtype=np.float64)
    prim = np.ascontiguousarray(prim)
    dp = ctypes.POINTER(ctypes.c_double)
    got = dev.dev_rest_max_speed(n, dx, bc, P.gamma, clean, ch, met.ctypes.data_as(dp), prim.ctypes.data_as(dp))
    want = O.max_speed(O.make_grid(P.n, P.dx, P.bc), O.make_opts(P.gamma, cleaning=bool(clean), ch=ch), met, prim)
    assert got > 0.0
    assert got == pytest.approx(want, rel=1e-13)
