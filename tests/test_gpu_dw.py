"""GPU parity of the double-word face path (precision HZ_FP64_DW: FP64 state, update, recovery and
CFL maximum; reconstruction, fluxes, HLLE, divergence and sources in pair-of-FP32 arithmetic)
against the FP64 oracle, at the FP64 bars: relative L1 per field <= 1e-10 after one step and
<= 1e-8 at end time."""
import numpy as np
import pytest

import oracle as O
from parity import (TOL_END, TOL_ONE_STEP, assert_parity, general_metric, gpu_run, gpu_solver,
                    oracle_run, oracle_setup, rel_l1)
from paper_1102_5202_gb300 import hzn
from paper_1102_5202_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DW = dict(precision=hzn.HZ_FP64_DW)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1102_5202_gb300 import build
    build.build_library()
    hzn.lib()


def _dt(P, cfl=0.5):
    grid, opts = oracle_setup(P)
    return cfl / O.max_speed(grid, opts, P.metric, P.prim)


@pytest.mark.parametrize("case", ["balsara1", "sod"])
def test_dw_tube_one_step(case):
    P = W.balsara1(400) if case == "balsara1" else W.sod(400)
    dt = _dt(P)
    gp, gc, gs = gpu_run(P, nsteps=1, dt=dt, solver=gpu_solver(P, **DW))
    op, oc, os_ = oracle_run(P, nsteps=1, dt=dt)
    assert gs["fails"] == 0 and os_["fails"] == 0
    assert_parity(gp, op, TOL_ONE_STEP, what=f"dw {case} prim")
    assert_parity(gc, oc, TOL_ONE_STEP, what=f"dw {case} cons")


def test_dw_balsara1_to_end_time():
    """Configuration 0 to t = 0.4 at CFL 0.5: the same number of steps as the oracle (the CFL
    maximum is FP64), end-time bar, and B^x exactly constant (its x flux is identically 0)."""
    P = W.balsara1(400)
    gp, gc, gs = gpu_run(P, t_end=0.4, cfl=0.5, solver=gpu_solver(P, **DW))
    op, oc, os_ = oracle_run(P, t_end=0.4, cfl=0.5)
    assert gs["steps"] == os_["steps"]
    assert abs(gs["t"] - 0.4) < 1e-14 and gs["fails"] == 0
    assert_parity(gp, op, TOL_END, what="dw balsara1 t=0.4 prim")
    assert_parity(gc, oc, TOL_END, what="dw balsara1 t=0.4 cons")
    assert np.all(gp[5] == 0.5)


def test_dw_max_speed_is_fp64():
    P = W.balsara1(400)
    s = gpu_solver(P, **DW)
    grid, opts = oracle_setup(P)
    assert s.max_speed() == pytest.approx(O.max_speed(grid, opts, P.metric, P.prim), rel=1e-13)


@pytest.mark.parametrize("dims,cleaning", [((37, 11, 7), False), ((37, 11, 7), True),
                                           ((70, 9, 1), True), ((33, 5, 66), False)])
def test_dw_curved_periodic_ragged(dims, cleaning):
    """General static metric (lapse, shift, non-diagonal gamma), periodic, ragged tiles."""
    P = W.smooth_periodic(dims, seed=5, amp=0.2, magnetised=True)
    P = W.with_periodic_metric(P, general_metric)
    if cleaning:
        P.cleaning, P.ch, P.kappa = True, 0.6, 0.7
        P.prim[8] = 0.01 * np.sin(np.arange(P.ncell).reshape(P.prim[8].shape) * 0.37)
    dt = _dt(P, 0.4)
    gp, gc, gs = gpu_run(P, nsteps=2, dt=dt, solver=gpu_solver(P, **DW))
    op, oc, os_ = oracle_run(P, nsteps=2, dt=dt)
    assert gs["fails"] == 0 and os_["fails"] == 0
    assert_parity(gp, op, TOL_ONE_STEP, what=f"dw {dims} prim", fields=range(9 if cleaning else 8))
    assert_parity(gc, oc, TOL_ONE_STEP, what=f"dw {dims} cons", fields=range(9 if cleaning else 8))


def test_dw_conservation_periodic():
    P = W.smooth_periodic((40, 24, 16), seed=9, amp=0.2, magnetised=True)
    dt = _dt(P, 0.4)
    s = gpu_solver(P, **DW)
    U0 = s.conserved().cpu().numpy()
    for _ in range(5):
        s.step(dt)
    U = s.conserved().cpu().numpy()
    d = (U - U0).reshape(9, -1).sum(1)
    scale = np.abs(U0).reshape(9, -1).sum(1)
    assert np.all(np.abs(d[:8]) <= 1e-13 * scale[:8])


def test_dw_blob_small_one_five_and_hundred_steps():
    """The benchmark's 3-D blob in the capped Schwarzschild metric at 40^3 (cleaning on), with
    its 1e-10 atmosphere (pressures near 1e-24: the FP32 exponent range is the pair's).  One step
    at the FP64 bar, five and a hundred steps at the end-time bar.  The pair path's faces carry
    48 significant bits against 53, and this case's oracle is well conditioned (a one-ulp input
    change moves it by <= 2e-12 after 100 steps): measured 1.3e-12 (one step), 5e-11 (five) and
    5.7e-11 (a hundred) in the worst field."""
    P = W.blob3d(40)
    dt = _dt(P)
    gp, gc, gs = gpu_run(P, nsteps=1, dt=dt, solver=gpu_solver(P, **DW))
    op, oc, os_ = oracle_run(P, nsteps=1, dt=dt)
    assert gs["fails"] == 0
    assert_parity(gp, op, TOL_ONE_STEP, what="dw blob40 1 step prim")
    assert_parity(gc, oc, TOL_ONE_STEP, what="dw blob40 1 step cons")
    for nsteps in (5, 100):
        gp, gc, gs = gpu_run(P, nsteps=nsteps, dt=dt, solver=gpu_solver(P, **DW))
        op, oc, os_ = oracle_run(P, nsteps=nsteps, dt=dt)
        assert gs["fails"] == os_["fails"] == 0
        assert_parity(gp, op, TOL_END, what=f"dw blob40 {nsteps} steps prim")
        assert_parity(gc, oc, TOL_END, what=f"dw blob40 {nsteps} steps cons")


def test_dw_against_fp64_gpu_blob64():
    """The pair path against the FP64 path itself, 3 steps of the 64^3 blob: the two differ by
    the pair's rounding only."""
    P = W.blob3d(64)
    dt = _dt(P)
    a, ac, _ = gpu_run(P, nsteps=3, dt=dt, solver=gpu_solver(P, **DW))
    b, bc, _ = gpu_run(P, nsteps=3, dt=dt, solver=gpu_solver(P))
    assert_parity(a, b, TOL_ONE_STEP, what="dw vs fp64 prim")
    assert_parity(ac, bc, TOL_ONE_STEP, what="dw vs fp64 cons")


def test_dw_atmosphere_threshold_and_floors():
    left = dict(rho=1.0, p=1.0)
    right = dict(rho=1e-13, p=1e-15)
    P = W.shock_tube(64, left, right, 5.0 / 3.0, 0.1)
    P.rho_floor, P.rho_atm, P.p_floor = 1e-13, 1e-11, 1e-16
    dt = 2e-3
    gp, gc, gs = gpu_run(P, nsteps=4, dt=dt, solver=gpu_solver(P, **DW))
    op, oc, os_ = oracle_run(P, nsteps=4, dt=dt)
    assert gs["fails"] == 0 and os_["fails"] == 0
    assert_parity(gp, op, TOL_ONE_STEP, what="dw atmosphere", fields=range(8))
    assert np.all(gp[0, 0, 0, -8:] == 1e-13) and np.all(gp[2, 0, 0, -8:] == 0.0)


def test_dw_rejects_ppm():
    P = W.balsara1(64)
    P.recon = 1
    with pytest.raises(hzn.HznError):
        gpu_solver(P, **DW)


def test_pair_arithmetic_error_bounds():
    """Each double-word operation of the pair path, run by the library on the GPU, against exact
    decimal arithmetic on the same pair inputs (bounds in dw_check.check_pair_results)."""
    import torch

    from dw_check import check_pair_results, pair_inputs

    a, b, m = pair_inputs()
    out = hzn.hz_dw_selftest(torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda"))
    check_pair_results(a, out.cpu().numpy(), m)
