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
    """At the surface of the blob the gas is cold (p/rho down to 1e-10), so its internal energy
    is below the FP32 resolution of the energy flux: a few surface cells can fail the recovery
    in mixed precision and are reset to the atmosphere.  They stay rare (<= 1e-3 of the cells)
    and the field errors stay within the stated bound."""
    P = W.blob3d(40)
    dt = _dt(P)
    # whole grid: the error sits in the ~200 near-vacuum cells next to the surface (rho 1e-11 to
    # 1e-7 beside rho 1e-4), where the FP32 rounding of the dense side's HLLE terms is as large
    # as the cell's own momentum; inside the star the FP32 path is accurate to ~1e-6
    # Over the whole grid only rho and p are compared: tenuous gas just above the atmosphere
    # threshold expands into the near vacuum and reaches Lorentz factors of tens within a few
    # steps in the FP64 oracle as well; its velocity is chaotic under any rounding difference.
    bound = {1: np.array([1e-5, 1e-5]), 5: np.array([1e-4, 1e-4])}
    for nsteps in (1, 5):
        gp, gc, gs = gpu_run(P, nsteps=nsteps, dt=dt, solver=_mixed(P))
        op, oc, _ = oracle_run(P, nsteps=nsteps, dt=dt)
        # failed recoveries (cells reset to the atmosphere), counted over all substeps
        assert gs["fails"] <= 1e-3 * P.ncell * 3 * nsteps
        r = rel_l1(gp, op)
        assert np.all(r[:2] <= bound[nsteps]), (nsteps, r)
        # the star's bulk: rho > 0.1 rho_max; B and psi carry the truncation-level divergence
        # error of the field's kink at p = 0.04 p_max, so their relative errors are larger
        star = op[0] > 0.1 * op[0].max()
        ri = rel_l1(gp[:, star][:, None, None, :], op[:, star][:, None, None, :])
        bulk = {1: np.array([1e-6, 1e-6, 5e-6, 5e-6, 5e-6, 1e-4, 1e-4, 2e-4, 1e-2]),
                5: np.array([1e-4, 1e-4, 2e-4, 2e-4, 2e-4, 1e-3, 1e-3, 1e-3, 5e-2])}[nsteps]
        assert np.all(ri <= bulk), (nsteps, ri)
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


def test_mixed_error_statement_96_100_steps():
    """The error statement of the mixed configuration at the oracle's size: blob 96^3, 100 CFL
    steps (the FP64 run's time steps replayed by the mixed run and the oracle), relative L1 per
    field.  Measured: FP64 GPU vs oracle <= 7e-12 in every field; mixed vs oracle, whole grid
    rho 1.2e-5, p 3.7e-6, u~ 3e-5..9e-5, B 1.9e-5, psi 2.4e-4; star bulk (rho > 0.1 max) 2e-6..4e-6,
    psi 2.6e-5."""
    import torch

    P = W.blob3d(96)
    s64 = hzn.Solver.for_problem(P)
    dts = []
    for _ in range(100):
        s64.step_cfl(0.5, 1e30)
        dts.append(s64.stats().dt)
    g64 = s64.primitives().cpu().numpy()
    assert s64.stats().c2p_failures == 0
    s64.close()
    s32 = _mixed(P)
    for dt in dts:
        s32.step(dt)
    g32 = s32.primitives().cpu().numpy()
    assert s32.stats().c2p_failures == 0
    s32.close()
    torch.cuda.synchronize()
    grid, opts = oracle_setup(P)
    U = O.grid_prim2cons(grid, opts, P.metric, P.prim)
    op = P.prim
    for dt in dts:
        op, U, nf = O.step(grid, opts, P.metric, op, U, dt)
        assert nf == 0
    r64 = rel_l1(g64, op)
    assert np.all(r64 <= 1e-10), r64
    r = rel_l1(g32, op)
    assert np.all(r <= np.array([5e-5, 2e-5, 3e-4, 3e-4, 2e-4, 1e-4, 1e-4, 1e-4, 1e-3])), r
    star = g64[0] > 0.1 * g64[0].max()
    rs = rel_l1(g32[:, star][:, None, None, :], op[:, star][:, None, None, :])
    assert np.all(rs <= np.array([2e-5] * 8 + [2e-4])), rs
    print(f"blob 96^3, 100 steps: FP64 GPU vs oracle max {r64.max():.1e}; mixed vs oracle whole grid "
          f"{np.array2string(r, precision=1)}; star bulk {np.array2string(rs, precision=1)}")
