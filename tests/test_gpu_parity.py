"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on identical seeded
inputs.  Bar (FP64): relative L1 per field <= 1e-10 after one step and <= 1e-8 at end time."""
import numpy as np
import pytest

import oracle as O
from parity import (TOL_END, TOL_ONE_STEP, assert_parity, general_metric, gpu_run, gpu_solver,
                    oracle_run, oracle_setup, rel_l1, tile_tube)
from paper_1102_5202_gb300 import hzn
from paper_1102_5202_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1102_5202_gb300 import build
    build.build_library()
    hzn.lib()


def _dt(P, cfl=0.5):
    grid, opts = oracle_setup(P)
    return cfl / O.max_speed(grid, opts, P.metric, P.prim)


# ------------------------------------------------------------------ 1-D tubes
@pytest.mark.parametrize("case", ["balsara1", "sod"])
def test_tube_one_step(case):
    P = W.balsara1(400) if case == "balsara1" else W.sod(400)
    dt = _dt(P)
    gp, gc, gs = gpu_run(P, nsteps=1, dt=dt)
    op, oc, os_ = oracle_run(P, nsteps=1, dt=dt)
    assert gs["fails"] == 0 and os_["fails"] == 0
    assert_parity(gp, op, TOL_ONE_STEP, what=f"{case} prim")
    assert_parity(gc, oc, TOL_ONE_STEP, what=f"{case} cons")


def test_balsara1_to_end_time():
    """Benchmark configuration 0: N = 400, Gamma = 2, CFL 0.5, t = 0.4, outflow."""
    P = W.balsara1(400)
    gp, gc, gs = gpu_run(P, t_end=0.4, cfl=0.5)
    op, oc, os_ = oracle_run(P, t_end=0.4, cfl=0.5)
    assert gs["steps"] == os_["steps"]
    assert abs(gs["t"] - 0.4) < 1e-14 and gs["fails"] == 0
    assert_parity(gp, op, TOL_END, what="balsara1 t=0.4 prim")
    assert_parity(gc, oc, TOL_END, what="balsara1 t=0.4 cons")
    assert np.all(gp[5] == 0.5)  # B^x stays exactly constant in 1-D


@pytest.mark.parametrize("case", ["blob_diag", "general_2d", "general_3d_cleaning"])
def test_device_cfl_rate_multi_d_matches_oracle(case):
    """The CFL rate in 2-D and 3-D (the sum over active axes of max|lambda|/dx, with the
    cleaning speed when on) on the device equals the oracle's, and the device's CFL step uses it."""
    if case == "blob_diag":
        P = W.blob3d(24)
    else:
        P = W.smooth_periodic((37, 11, 7) if case.endswith("3d_cleaning") else (70, 9, 1), seed=5,
                              amp=0.2, magnetised=True)
        P = W.with_periodic_metric(P, general_metric)
        if case.endswith("cleaning"):
            P.cleaning, P.ch, P.kappa = True, 0.9, 0.7
    s = gpu_solver(P)
    grid, opts = oracle_setup(P)
    want = O.max_speed(grid, opts, P.metric, P.prim)
    assert s.max_speed() == pytest.approx(want, rel=1e-13)
    s.step_cfl(0.5, 1e30)
    assert s.stats().dt == pytest.approx(0.5 / want, rel=1e-13)


def test_device_cfl_matches_oracle_dt():
    P = W.balsara1(400)
    s = gpu_solver(P)
    grid, opts = oracle_setup(P)
    want = O.max_speed(grid, opts, P.metric, P.prim)
    assert s.max_speed() == pytest.approx(want, rel=1e-13)
    s.step_cfl(0.5, 0.4)
    st = s.stats()
    assert st.dt == pytest.approx(0.5 / want, rel=1e-13) and st.steps == 1


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_tube_along_each_axis(axis):
    """The same tube along x, y or z (transverse axes periodic, 3 cells: ragged tiles)."""
    P1 = W.balsara1(96)
    P = tile_tube(P1, axis, other=3)
    dt = _dt(P)
    gp, gc, _ = gpu_run(P, nsteps=3, dt=dt)
    op, oc, _ = oracle_run(P, nsteps=3, dt=dt)
    assert_parity(gp, op, TOL_ONE_STEP, what=f"axis {axis}")
    # direction symmetry of the GPU path itself
    ref, _, _ = gpu_run(P1, nsteps=3, dt=dt)
    perm = [(0, 1, 2), (1, 2, 0), (2, 0, 1)][axis]
    line = {0: lambda a: a[:, 0, 0, :], 1: lambda a: a[:, 0, :, 0], 2: lambda a: a[:, :, 0, 0]}[axis](gp)
    back = line.copy()
    for k in range(3):
        back[2 + k] = line[2 + perm[k]]
        back[5 + k] = line[5 + perm[k]]
    assert np.allclose(back, ref[:, 0, 0, :], rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------------ multi-D, curved metric
@pytest.mark.parametrize("dims,cleaning", [((37, 11, 7), False), ((37, 11, 7), True),
                                           ((70, 9, 1), True), ((33, 5, 66), False)])
def test_curved_periodic_ragged(dims, cleaning):
    """General static metric (lapse, shift, non-diagonal gamma), periodic, several tiles with
    ragged tails in every direction, z chunks; with and without cleaning."""
    P = W.smooth_periodic(dims, seed=5, amp=0.2, magnetised=True)
    P = W.with_periodic_metric(P, general_metric)
    if cleaning:
        P.cleaning, P.ch, P.kappa = True, 0.6, 0.7
        P.prim[8] = 0.01 * np.sin(np.arange(P.ncell).reshape(P.prim[8].shape) * 0.37)
    dt = _dt(P, 0.4)
    gp, gc, gs = gpu_run(P, nsteps=2, dt=dt)
    op, oc, os_ = oracle_run(P, nsteps=2, dt=dt)
    assert gs["fails"] == 0 and os_["fails"] == 0
    assert_parity(gp, op, TOL_ONE_STEP, what=f"{dims} prim", fields=range(9 if cleaning else 8))
    assert_parity(gc, oc, TOL_ONE_STEP, what=f"{dims} cons", fields=range(9 if cleaning else 8))


def test_conservation_periodic_gpu():
    P = W.smooth_periodic((40, 24, 16), seed=9, amp=0.2, magnetised=True)
    dt = _dt(P, 0.4)
    s = gpu_solver(P)
    U0 = s.conserved().cpu().numpy()
    for _ in range(5):
        s.step(dt)
    U = s.conserved().cpu().numpy()
    d = (U - U0).reshape(9, -1).sum(1)
    scale = np.abs(U0).reshape(9, -1).sum(1)
    assert np.all(np.abs(d[:8]) <= 1e-13 * scale[:8])


# ------------------------------------------------------------------ 3-D blob (benchmark setup)
def test_blob_small_one_and_five_steps():
    """The benchmark's 3-D blob in the capped Schwarzschild metric at 40^3 (cleaning on)."""
    P = W.blob3d(40)
    dt = _dt(P)
    gp, gc, gs = gpu_run(P, nsteps=1, dt=dt)
    op, oc, os_ = oracle_run(P, nsteps=1, dt=dt)
    assert_parity(gp, op, TOL_ONE_STEP, what="blob40 1 step prim")
    assert_parity(gc, oc, TOL_ONE_STEP, what="blob40 1 step cons")
    gp, gc, gs = gpu_run(P, nsteps=5, dt=dt)
    op, oc, os_ = oracle_run(P, nsteps=5, dt=dt)
    assert_parity(gp, op, TOL_END, what="blob40 5 steps prim")
    assert_parity(gc, oc, TOL_END, what="blob40 5 steps cons")


def test_blob_full_size_sampled():
    """Full benchmark size (192^3, one step at the CFL dt): sampled cells against the oracle run
    on the 13^3 neighbourhood that determines them (3 substeps x 2-cell stencil)."""
    import torch

    P = W.blob3d(192)
    s = gpu_solver(P)
    vmax = s.max_speed()
    dt = 0.5 / vmax
    s.step(dt)
    gp = s.primitives().cpu().numpy()
    st = s.stats()
    assert st.c2p_failures == 0
    rng = np.random.Generator(np.random.PCG64(77))
    n = P.n[0]
    # cells in the star, near its surface, in the atmosphere and at the domain boundary
    picks = [(96, 96, 96), (100, 90, 70), (96, 96 + 38, 96), (5, 100, 100), (0, 0, 0), (191, 50, 191)]
    picks += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(10)]
    m = 6
    fscale = np.maximum(np.abs(P.prim.reshape(9, -1)).max(axis=1), np.abs(gp.reshape(9, -1)).max(axis=1))
    for (i, j, k) in picks:
        lo = [max(0, c - m) for c in (i, j, k)]
        hi = [min(n, c + m + 1) for c in (i, j, k)]
        Q = P.subbox(lo, hi)
        op, _, _ = oracle_run(Q, nsteps=1, dt=dt)
        got = gp[:, k, j, i]
        want = op[:, k - lo[2], j - lo[1], i - lo[0]]
        err = np.abs(got - want) / np.maximum(fscale, 1e-300)
        assert np.all(err <= 1e-10), ((i, j, k), err)
    torch.cuda.synchronize()


# ------------------------------------------------------------------ edge cases
def test_atmosphere_threshold_and_floors():
    """Expansion into a near vacuum: the right state sits below the atmosphere threshold, so
    those cells are set to the atmosphere on both sides without a recovery; the expanding gas
    crosses the threshold and the pressure floor as it goes."""
    left = dict(rho=1.0, p=1.0)
    right = dict(rho=1e-13, p=1e-15)
    P = W.shock_tube(64, left, right, 5.0 / 3.0, 0.1)
    P.rho_floor, P.rho_atm, P.p_floor = 1e-13, 1e-11, 1e-16
    dt = 2e-3
    gp, gc, gs = gpu_run(P, nsteps=4, dt=dt)
    op, oc, os_ = oracle_run(P, nsteps=4, dt=dt)
    assert gs["fails"] == 0 and os_["fails"] == 0
    assert_parity(gp, op, TOL_ONE_STEP, what="atmosphere", fields=range(8))
    assert np.all(gp[0, 0, 0, -8:] == 1e-13) and np.all(gp[2, 0, 0, -8:] == 0.0)


def test_recovery_fallback_hard_states():
    """Pointwise recovery of hard states (W up to 10, b^2/rho up to 100, random metric) from a
    poor initial guess through the step: a uniform periodic box of each state is stationary, so
    one step must return it unchanged (to round-off) whichever Newton path was taken."""
    n = 64
    met = W.random_metric_points(n, seed=61)
    prim = W.random_prim_points(n, seed=62, met=met, wmax=10.0, sigma_max=100.0)
    for c in range(0, n, 8):
        P = W.Problem("u", (4, 1, 1), (0.1, 1.0, 1.0), (0, 0, 0), (1, 1, 1), 5.0 / 3.0,
                      np.ascontiguousarray(np.repeat(prim[c][:, None, None, None], 4, axis=3)),
                      np.ascontiguousarray(np.repeat(met[c][:, None, None, None], 6, axis=3)))
        gp, gc, gs = gpu_run(P, nsteps=1, dt=1e-3)
        assert gs["fails"] == 0
        scale = np.abs(prim[c]).max()
        assert np.abs(gp[:, 0, 0, 0] - prim[c]).max() <= 1e-9 * max(scale, 1.0), c


def test_state_calls_out_of_order():
    s = hzn.Solver((16, 1, 1), (0.1, 1, 1), (0, 0, 0), hzn.make_options(2.0))
    with pytest.raises(hzn.HznError) as e:
        s.step(0.01)
    assert e.value.code == hzn.HZ_ERR_STATE
    with pytest.raises(hzn.HznError):
        s.set_primitives(np.zeros((9, 1, 1, 16)))  # metric first


def test_fp64_reciprocal_error_bound():
    """The FP64 kernels' reciprocal (hardware approximation + two Newton-Raphson steps) against
    the correctly rounded 1/x over normal x of both signs across the exponent range, and on
    powers of two (exact): within 2 ulps."""
    import torch

    rng = np.random.Generator(np.random.PCG64(91))
    e = rng.uniform(-1000.0, 1000.0, 200000)
    x = np.ldexp(rng.uniform(1.0, 2.0, e.size), e.astype(np.int64)) * rng.choice([-1.0, 1.0], e.size)
    x = np.concatenate([x, np.ldexp(1.0, np.arange(-1000, 1001)), [1.0, -1.0, 3.0, 1.0 / 3.0]])
    got = hzn.hz_rcp_selftest(torch.tensor(x, device="cuda")).cpu().numpy()
    want = 1.0 / x
    ulps = np.abs(got - want) / np.spacing(np.abs(want))
    assert ulps.max() <= 2.0, ulps.max()
    p2 = np.ldexp(1.0, np.arange(-1000, 1001))
    assert np.all(hzn.hz_rcp_selftest(torch.tensor(p2, device="cuda")).cpu().numpy() == 1.0 / p2)
