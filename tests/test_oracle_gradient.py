"""Pins of the oracle's complex-step derivative (the FP64 gradient reference of the adjoint).

The oracle runs the scheme on complex primitives P + i h dP with every branch decision (limiter,
wave-speed bounds, floors) taken on the real part; Im(result) / h is then the derivative of the
discrete update in the direction dP.  These tests pin it to what the mathematics fixes, not to
itself: central finite differences, linearity in the direction, conservation of the derivative
of a conserved total in a periodic box, and the real part equal to the plain FP64 run."""
import numpy as np
import pytest

from parity import oracle_setup
from paper_1102_5202_gb300 import workloads as W
import oracle as O


def _fd(P, grid, opts, dprim, eps, dt, nsteps):
    out = []
    for s in (+1.0, -1.0):
        p = P.prim + s * eps * dprim
        u = O.grid_prim2cons(grid, opts, P.metric, p)
        out.append(O.evolve(grid, opts, P.metric, p, u, 1e30, 0.0, fixed_dt=dt, max_steps=nsteps)[0])
    return (out[0] - out[1]) / (2.0 * eps)


def _tube(n=120, noise=1e-3, seed=1104):
    """Shock tube of the default states with a small seeded texture on every field but B^x, so
    that no limiter or wave-speed decision sits on or near a tie (a uniform state puts every
    slope on the kink of |x|, where only directions uniform across the state are
    differentiable)."""
    P = W.balsara1(n)
    if noise:
        rng = np.random.default_rng(seed)
        P.prim = P.prim.copy()
        for f in (0, 1):
            P.prim[f] *= 1.0 + noise * rng.standard_normal(P.prim[f].shape)
        for f in (2, 3, 4, 6, 7):  # every field but B^x, which must stay uniform
            P.prim[f] += noise * rng.standard_normal(P.prim[f].shape)
    grid, opts = oracle_setup(P)
    dt = 0.4 / O.max_speed(grid, opts, P.metric, P.prim)
    return P, grid, opts, dt


def test_complex_step_matches_central_differences():
    P, grid, opts, dt = _tube()
    rng = np.random.default_rng(7)
    dprim = np.zeros_like(P.prim)
    x = (np.arange(P.n[0]) + 0.5) / P.n[0]
    # left-state pressure scale, a smooth density perturbation, per-cell B^y noise
    dprim[1, ..., : P.n[0] // 2] = P.prim[1, ..., : P.n[0] // 2]
    dprim[0] = 0.3 * P.prim[0] * np.sin(2 * np.pi * x)
    dprim[6] = 0.1 * rng.standard_normal(P.prim[6].shape) * np.abs(P.prim[6])
    _, dcs, _, _, nf = O.evolve_cs(grid, opts, P.metric, P.prim, dprim, 1e-30, dt, 30)
    assert nf == 0
    # a step of 1e-8 keeps branch crossings (which vanish as the step shrinks) below the
    # round-off of the difference quotient, about 1e-16 / 1e-8 relative
    dfd = _fd(P, grid, opts, dprim, 1e-8, dt, 30)
    for f in range(8):
        den = np.abs(dcs[f]).sum()
        if den == 0.0:
            assert np.abs(dfd[f]).max() < 1e-8
            continue
        assert np.abs(dfd[f] - dcs[f]).sum() / den < 2e-6, (f, np.abs(dfd[f] - dcs[f]).sum() / den)


def test_uniform_state_direction_is_frozen_at_the_kink():
    """On a uniform state every limited slope sits on the kink of |x|: the frozen-branch
    derivative keeps the slope at zero, so a perturbation of one uniform region that is not
    itself uniform gives a derivative that differs from central differences, while a uniform
    rescaling of the region agrees with them."""
    P, grid, opts, dt = _tube(noise=0.0)
    n = P.n[0]
    uni = np.zeros_like(P.prim)
    uni[1, ..., : n // 2] = P.prim[1, ..., : n // 2]
    _, dcs, _, _, _ = O.evolve_cs(grid, opts, P.metric, P.prim, uni, 1e-30, dt, 20)
    dfd = _fd(P, grid, opts, uni, 1e-6, dt, 20)
    assert np.abs(dfd[0] - dcs[0]).sum() / np.abs(dcs[0]).sum() < 1e-7
    x = (np.arange(n) + 0.5) / n
    bump = np.zeros_like(P.prim)
    bump[0] = P.prim[0] * np.sin(2 * np.pi * x) * (x > 0.5)
    _, dcs, _, _, _ = O.evolve_cs(grid, opts, P.metric, P.prim, bump, 1e-30, dt, 20)
    dfd = _fd(P, grid, opts, bump, 1e-6, dt, 20)
    assert np.abs(dfd[0] - dcs[0]).sum() / np.abs(dcs[0]).sum() > 1e-3


def test_complex_step_is_linear_in_the_direction():
    P, grid, opts, dt = _tube(80)
    rng = np.random.default_rng(3)
    d1 = rng.standard_normal(P.prim.shape) * P.prim * 0.1
    d2 = rng.standard_normal(P.prim.shape) * P.prim * 0.1
    d1[8] = d2[8] = 0.0
    d1[5] = d2[5] = 0.0  # B^x uniform: a jump would violate the constraint
    a, b = 0.7, -1.9
    _, g1, _, _, _ = O.evolve_cs(grid, opts, P.metric, P.prim, d1, 1e-30, dt, 10)
    _, g2, _, _, _ = O.evolve_cs(grid, opts, P.metric, P.prim, d2, 1e-30, dt, 10)
    _, g12, _, _, _ = O.evolve_cs(grid, opts, P.metric, P.prim, a * d1 + b * d2, 1e-30, dt, 10)
    ref = a * g1 + b * g2
    assert np.abs(g12 - ref).max() <= 1e-11 * np.abs(ref).max()


def test_real_part_is_the_fp64_run():
    P, grid, opts, dt = _tube(80)
    dprim = np.zeros_like(P.prim)
    dprim[0] = P.prim[0]
    pre, _, _, _, _ = O.evolve_cs(grid, opts, P.metric, P.prim, dprim, 1e-30, dt, 10)
    u = O.grid_prim2cons(grid, opts, P.metric, P.prim)
    ref = O.evolve(grid, opts, P.metric, P.prim, u, 1e30, 0.0, fixed_dt=dt, max_steps=10)[0]
    assert np.abs(pre - ref).max() <= 1e-13 * np.abs(ref).max()


def test_derivative_of_conserved_totals_is_conserved():
    """Periodic box, no source (Minkowski), no floors touched: sum over cells of every conserved
    component is constant in time (§2.1 Eq. 2 in conservation form), hence so is its derivative."""
    P = W.smooth_periodic((24, 10, 1), seed=11, amp=0.2, magnetised=True)
    grid, opts = oracle_setup(P)
    dt = 0.4 / O.max_speed(grid, opts, P.metric, P.prim)
    rng = np.random.default_rng(5)
    dprim = rng.standard_normal(P.prim.shape) * 0.05 * np.abs(P.prim).max(axis=(1, 2, 3))[:, None, None, None]
    dprim[8] = 0.0
    dprim[5:8] = 0.0  # keep the field divergence-free
    _, _, ce, dce, nf = O.evolve_cs(grid, opts, P.metric, P.prim, dprim, 1e-30, dt, 6)
    assert nf == 0
    _, _, c0, dc0, _ = O.evolve_cs(grid, opts, P.metric, P.prim, dprim, 1e-30, dt, 0)
    for f in range(8):
        scale = np.abs(dc0[f]).sum() + np.abs(dce[f]).sum() + 1e-300
        assert abs(dce[f].sum() - dc0[f].sum()) <= 1e-12 * scale, f


@pytest.mark.parametrize("h", [1e-30, 1e-200])
def test_step_size_independence(h):
    """No difference of nearby values is formed, so the result does not depend on h."""
    P, grid, opts, dt = _tube(60)
    dprim = np.zeros_like(P.prim)
    dprim[1] = P.prim[1]
    _, g, _, _, _ = O.evolve_cs(grid, opts, P.metric, P.prim, dprim, h, dt, 5)
    _, gref, _, _, _ = O.evolve_cs(grid, opts, P.metric, P.prim, dprim, 1e-20, dt, 5)
    assert np.abs(g - gref).max() <= 1e-12 * np.abs(gref).max()
