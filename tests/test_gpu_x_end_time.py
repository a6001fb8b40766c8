"""End-time parity on the benchmark's 3-D blob (the update of §2.1 Eq. 2 with the scheme of §2.2
and §3.2, on the stand-in for the rotating star of §4.1 and §5.2): the FP64 and mixed-precision
paths against the FP64 oracle after 100 CFL steps.  This file is collected after the parity
suites (test_gpu_parity.py, test_gpu_variants.py), so that a run stopping at its first failure
has run those first.

Conditioning of the workload (measured on the oracle alone, CPU):
  * 40^3: a one-ulp change of the input moves the oracle's own result by <= 2e-12 (relative L1
    per field) after 100 steps, so the end-time bar of the benchmark statement, 1e-8, applies
    as it stands (GPU vs oracle measured 1.6e-12).
  * 96^3: the near-vacuum gas at the star's surface (rho from 1e-13 to 1e-8 beside 1e-4, p/rho
    below 1e-8, ~2,600 cells at the pressure floor) amplifies a one-ulp input change to 1e-7 ..
    1e-4 relative within a few steps; then a discrete decision flips.  At step 9, stage 1, cell
    (28, 45, 47) has D / sqrt(gamma) = 1.28023e-12 against the atmosphere threshold 1.28e-12 in
    one run and lies below it in the other: one run keeps the cell, the other resets it to the
    atmosphere.  That O(1) change of one cell then spreads into the star as a small wave.  After
    100 steps the oracle differs from itself by up to 8e-8 (rho) .. 2e-6 (psi) relative L1,
    depending on which perturbation flips which cell first (rho +1 ulp, p -1 ulp, every field
    +-1 ulp: rho 7.8e-8 / 1.2e-9 / 1.1e-8).  The GPU path meets the same flip: at step 10 its
    distance from the oracle equals the rho +1 ulp run's to three digits, and after 100 steps it
    is within 1.35x of that run in every field.
So at 96^3 the end-time check is: the first five steps (before any flip) at 1e-8; after 100
steps, every field within SPREAD_FACTOR x the oracle's own spread over three one-ulp
perturbations, and the grid integrals of the conserved fields (which one cell's flip barely
moves) within the same factor of their spread.
"""
import numpy as np
import pytest

from parity import (SPREAD_FACTOR, TOL_END, assert_parity, assert_within_spread, integral_diff,
                    oracle_replay, oracle_setup, perturbed, rel_l1)
from paper_1102_5202_gb300 import hzn
from paper_1102_5202_gb300 import workloads as W
import oracle as O

pytestmark = pytest.mark.gpu

EARLY = 5  # steps compared at the plain end-time bar (the first flip comes at step 9)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1102_5202_gb300 import build
    build.build_library()
    hzn.lib()


def _gpu_cfl_run(P, nsteps, precision=hzn.HZ_FP64, keep=()):
    """nsteps device-CFL steps; returns (prim, cons, dts, {step: prim}, failures)."""
    s = hzn.Solver.for_problem(P, precision=precision)
    dts, kept = [], {}
    for k in range(1, nsteps + 1):
        s.step_cfl(0.5, 1e30)
        dts.append(s.stats().dt)
        if k in keep:
            kept[k] = s.primitives().cpu().numpy()
    prim, cons = s.primitives().cpu().numpy(), s.conserved().cpu().numpy()
    fails = s.stats().c2p_failures
    s.close()
    return prim, cons, dts, kept, fails


def test_blob40_fp64_100_cfl_steps_at_the_end_time_bar():
    """40^3, 100 CFL steps (the GPU's time steps replayed by the oracle): every primitive and
    conserved field within 1e-8 relative L1 (measured 1.6e-12), and the oracle's own one-ulp
    spread far below it."""
    P = W.blob3d(40)
    g, gc, dts, _, fails = _gpu_cfl_run(P, 100)
    assert fails == 0
    op, oc = oracle_replay(P, dts)
    assert_parity(g, op, TOL_END, what="blob40 100 steps prim")
    assert_parity(gc, oc, TOL_END, what="blob40 100 steps cons")
    sp = rel_l1(oracle_replay(perturbed(P, "rho"), dts)[0], op)
    assert np.all(sp <= 1e-3 * TOL_END), sp


@pytest.fixture(scope="module")
def blob96():
    import torch

    P = W.blob3d(96)
    g, gc, dts, kept, fails = _gpu_cfl_run(P, 100, keep=(EARLY,))
    # the mixed path over the FP64 run's time steps
    s = hzn.Solver.for_problem(P, precision=hzn.HZ_MIXED)
    for dt in dts:
        s.step(dt)
    g32, f32 = s.primitives().cpu().numpy(), s.stats().c2p_failures
    s.close()
    torch.cuda.synchronize()
    grid, opts = oracle_setup(P)
    U = O.grid_prim2cons(grid, opts, P.metric, P.prim)
    op, early = P.prim, None
    for k, dt in enumerate(dts, 1):
        op, U, nf = O.step(grid, opts, P.metric, op, U, dt)
        assert nf == 0
        if k == EARLY:
            early = op
    runs = {kind: oracle_replay(perturbed(P, kind), dts) for kind in ("rho", "p", "all")}
    return dict(P=P, dts=dts, g=g, gc=gc, g_early=kept[EARLY], fails=fails, g32=g32, f32=f32,
                op=op, oc=U, op_early=early, runs=runs)


def test_blob96_fp64_first_steps_at_the_end_time_bar(blob96):
    assert blob96["fails"] == 0
    assert_parity(blob96["g_early"], blob96["op_early"], TOL_END, what=f"blob96 {EARLY} steps")


def test_blob96_fp64_100_steps_within_the_oracles_spread(blob96):
    op, oc = blob96["op"], blob96["oc"]
    spread = np.zeros(9)
    ispread = np.zeros(9)
    for prim, cons in blob96["runs"].values():
        spread = np.maximum(spread, rel_l1(prim, op))
        ispread = np.maximum(ispread, integral_diff(cons, oc))
    r, bar = assert_within_spread(blob96["g"], op, spread, what="blob96 100 steps")
    gi = integral_diff(blob96["gc"], oc)
    ibar = np.maximum(1e-15, SPREAD_FACTOR * ispread)
    assert np.all(gi <= ibar), (gi, ibar)
    # the flips leave the conserved totals alone: mass to 1e-12, energy to 1e-10
    assert gi[0] <= 1e-12 and gi[1] <= 1e-10, gi
    print(f"blob 96^3, 100 steps: FP64 GPU vs oracle {np.array2string(r, precision=1)}; "
          f"oracle spread {np.array2string(spread, precision=1)}; integrals {np.array2string(gi, precision=1)}")


def test_blob96_mixed_error_statement(blob96):
    """The error statement of the mixed configuration at the oracle's size: blob 96^3, 100 CFL
    steps (the FP64 run's time steps replayed by the mixed run and the oracle), relative L1 per
    field.  Measured: whole grid rho 1.3e-5, p 6.1e-6, u~ 3.4e-5 .. 5.6e-5, B 1.5e-5 .. 2.2e-5,
    psi 4.0e-4; star bulk (rho > 0.1 max) rho 4.0e-6, p 3.3e-6, u~ 6.6e-6 .. 9.5e-6, B 4.6e-6 ..
    7.7e-6, psi 9.3e-5.  These are 100x and more above the oracle's own spread (the FP32 faces
    set them), so they are compared directly."""
    g32, op = blob96["g32"], blob96["op"]
    assert blob96["f32"] == 0
    r = rel_l1(g32, op)
    assert np.all(r <= np.array([5e-5, 2e-5, 3e-4, 3e-4, 2e-4, 1e-4, 1e-4, 1e-4, 1e-3])), r
    star = op[0] > 0.1 * op[0].max()
    rs = rel_l1(g32[:, star][:, None, None, :], op[:, star][:, None, None, :])
    assert np.all(rs <= np.array([2e-5] * 8 + [2e-4])), rs
    print(f"blob 96^3, 100 steps: mixed vs oracle whole grid {np.array2string(r, precision=1)}; "
          f"star bulk {np.array2string(rs, precision=1)}")
