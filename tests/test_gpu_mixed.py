"""Mixed precision (FP32 reconstruction, fluxes and sources with FP32 flux-divergence
accumulation; FP64 conserved state, RK update, recovery and CFL maximum) against the FP64
oracle on identical seeded inputs.  The bar is the error the FP32 face arithmetic implies
(relative L1 per field, stated in each test), well below the scheme's truncation error; the
paper's own single- versus double-precision differences are of the same order (§5.1-§5.3)."""
import numpy as np
import pytest

from parity import assert_parity, gpu_run, oracle_run, oracle_setup, rel_l1
from paper_1102_5202_gb300 import hzn
from paper_1102_5202_gb300 import workloads as W
import oracle as O

pytestmark = pytest.mark.gpu

TOL_MIXED_ONE_STEP = 2e-6
TOL_MIXED_END = 5e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1102_5202_gb300 import build
    build.build_library()
    hzn.lib()


def _dt(P, cfl=0.5):
    grid, opts = oracle_setup(P)
    return cfl / O.max_speed(grid, opts, P.metric, P.prim)


def _mixed(P):
    return hzn.Solver.for_problem(P, precision=hzn.HZ_MIXED)


@pytest.mark.parametrize("case", ["balsara1", "sod"])
def test_mixed_tube_one_step_and_end(case):
    P = W.balsara1(400) if case == "balsara1" else W.sod(400)
    dt = _dt(P)
    gp, _, gs = gpu_run(P, nsteps=1, dt=dt, solver=_mixed(P))
    op, _, _ = oracle_run(P, nsteps=1, dt=dt)
    assert gs["fails"] == 0
    r1 = assert_parity(gp, op, TOL_MIXED_ONE_STEP, fields=range(8), what=f"{case} mixed 1 step")
    gp, _, gs = gpu_run(P, t_end=0.4, cfl=0.5, solver=_mixed(P))
    op, _, os_ = oracle_run(P, t_end=0.4, cfl=0.5)
    r2 = assert_parity(gp, op, TOL_MIXED_END, fields=range(8), what=f"{case} mixed t=0.4")
    print(f"{case} mixed vs FP64 oracle, relative L1 per field: 1 step {np.array2string(r1[:8], precision=1)}"
          f"; t=0.4 {np.array2string(r2[:8], precision=1)}")


def test_mixed_blob_one_and_five_steps():
    """The blob at 40^3 after one and five steps, every field over the whole grid and over the
    star's bulk (rho > 0.1 rho_max).  Measured (relative L1 per field, rho p u~x u~y u~z Bx By Bz
    psi): whole grid after one step 7.8e-7 1.5e-7 3.3e-3 3.9e-3 2.4e-4 1.4e-5 1.4e-5 1.8e-5
    6.3e-4, after five 6.4e-6 1.8e-6 3.6e-3 3.4e-3 9.0e-4 2.1e-5 1.9e-5 2.0e-5 6.3e-4; bulk
    <= 1.2e-5 (psi 1.8e-4).  The whole-grid velocity error sits in the near-vacuum cells next to
    the surface (rho 1e-11 .. 1e-7 beside 1e-4): the FP32 face arithmetic resolves the dense
    neighbour's momentum flux to 6e-8 of itself, which in a cell 1e4 .. 1e7 times less dense is
    a velocity change of order one.  It is the FP32 faces' own error, not conditioning: the
    oracle run from the FP32-rounded input differs from the oracle by <= 4e-8 in u~."""
    P = W.blob3d(40)
    dt = _dt(P)
    whole = {1: np.array([1e-5, 1e-5, 1e-2, 1e-2, 1e-2, 1e-4, 1e-4, 1e-4, 5e-3]),
             5: np.array([1e-4, 1e-4, 1e-2, 1e-2, 1e-2, 1e-4, 1e-4, 1e-4, 5e-3])}
    bulk = {1: np.array([1e-6, 1e-6, 5e-6, 5e-6, 5e-6, 1e-4, 1e-4, 2e-4, 1e-2]),
            5: np.array([1e-4, 1e-4, 2e-4, 2e-4, 2e-4, 1e-3, 1e-3, 1e-3, 5e-2])}
    for nsteps in (1, 5):
        gp, gc, gs = gpu_run(P, nsteps=nsteps, dt=dt, solver=_mixed(P))
        op, oc, _ = oracle_run(P, nsteps=nsteps, dt=dt)
        # failed recoveries (cells reset to the atmosphere), counted over all substeps
        assert gs["fails"] <= 1e-3 * P.ncell * 3 * nsteps
        r = rel_l1(gp, op)
        assert np.all(r <= whole[nsteps]), (nsteps, r)
        star = op[0] > 0.1 * op[0].max()
        ri = rel_l1(gp[:, star][:, None, None, :], op[:, star][:, None, None, :])
        assert np.all(ri <= bulk[nsteps]), (nsteps, ri)
        print(f"blob40 mixed vs FP64 oracle after {nsteps} step(s): all cells "
              f"{np.array2string(r, precision=1)}; star bulk (rho > 0.1 max) {np.array2string(ri, precision=1)}")


def test_mixed_general_metric_periodic():
    from parity import general_metric

    P = W.smooth_periodic((37, 11, 7), seed=5, amp=0.2, magnetised=True)
    P = W.with_periodic_metric(P, general_metric)
    P.cleaning, P.ch, P.kappa = True, 0.6, 0.7
    dt = _dt(P, 0.4)
    gp, _, gs = gpu_run(P, nsteps=2, dt=dt, solver=_mixed(P))
    op, _, _ = oracle_run(P, nsteps=2, dt=dt)
    assert gs["fails"] == 0
    assert_parity(gp, op, TOL_MIXED_ONE_STEP, what="general metric mixed")


def test_diag_and_general_kernels_agree():
    """The same diagonal metric through the zero-shift kernel and, with a shift of 1e-300 in
    one ghost cell forcing the general kernel, gives the same result to round-off."""
    P = W.blob3d(24)
    Q = W.blob3d(24)
    Q.metric = Q.metric.copy()
    Q.metric[1, 0, 0, 0] = 1e-300
    dt = _dt(P)
    a, _, _ = gpu_run(P, nsteps=2, dt=dt)
    b, _, _ = gpu_run(Q, nsteps=2, dt=dt)
    assert np.all(rel_l1(a, b) <= 1e-12)


def _diag_metric(X, Y, Z):
    """A smooth periodic static metric with zero shift and diagonal gamma_ij (the class the
    zero-shift kernels take)."""
    from parity import general_metric

    m = general_metric(X, Y, Z)
    m[1:4] = 0.0
    m[5] = m[6] = m[8] = 0.0
    return m


@pytest.mark.parametrize("n", [(37, 11, 7), (33, 2, 5), (2, 6, 3)])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("clean", [True, False])
def test_mixed_3d_staged_plane_tiles(n, bc, clean):
    """The mixed 3-D kernel reads the stencils of its x and y faces from a primitive plane staged
    in shared memory (the tile with a two-cell halo, boundary indices resolved when the plane is
    copied in): ragged tiles in x and y, two-cell axes, outflow and periodic boundaries, with and
    without cleaning, on a zero-shift diagonal metric, against the oracle at the mixed one-step
    bar over two steps."""
    P = W.smooth_periodic(n, seed=11, amp=0.2, magnetised=True)
    P = W.with_periodic_metric(P, _diag_metric)
    P.bc = (bc, bc, bc)
    if clean:
        P.cleaning, P.ch, P.kappa = True, 0.6, 0.7
    dt = _dt(P, 0.4)
    gp, _, gs = gpu_run(P, nsteps=2, dt=dt, solver=_mixed(P))
    op, _, _ = oracle_run(P, nsteps=2, dt=dt)
    assert gs["fails"] == 0
    assert_parity(gp, op, TOL_MIXED_ONE_STEP, fields=range(9 if clean else 8),
                  what=f"staged mixed {n} bc={bc} clean={clean}")


@pytest.mark.parametrize("axis", [0, 2])
def test_mixed_atmosphere_threshold_and_floors(axis):
    """The mixed path's resets: expansion into a near vacuum (the right state below the
    atmosphere threshold; the expanding gas crosses the threshold and the density and pressure
    floors, so recovered cells are reset after the iteration, which rewrites their conserved
    vector), along x in 2-D and along z in 3-D, against the oracle at the mixed one-step bar."""
    from parity import tile_tube

    left = dict(rho=1.0, p=1.0)
    right = dict(rho=1e-13, p=1e-15)
    P = tile_tube(W.shock_tube(64, left, right, 5.0 / 3.0, 0.1), axis)
    P.rho_floor, P.rho_atm, P.p_floor = 1e-13, 1e-11, 1e-16
    dt = 2e-3
    gp, gc, gs = gpu_run(P, nsteps=4, dt=dt, solver=_mixed(P))
    op, oc, os_ = oracle_run(P, nsteps=4, dt=dt)
    assert gs["fails"] == 0 and os_["fails"] == 0
    assert_parity(gp, op, TOL_MIXED_ONE_STEP, fields=range(8), what=f"mixed atmosphere axis {axis}")
    # conserved vector too: a reset cell's rewritten U is what the oracle's reset gives
    assert_parity(gc, oc, TOL_MIXED_ONE_STEP, fields=range(8), what=f"mixed atmosphere U axis {axis}")
    tail = gp[0].reshape(-1, 64)[:, -8:] if axis == 0 else gp[0].reshape(64, -1)[-8:]
    assert np.allclose(tail, 1e-13, rtol=1e-7, atol=0)
