"""Helpers of the GPU-vs-oracle parity tests: run the same seeded problem through the C-ABI
(CUDA) and through the FP64 oracle, and compare field by field."""
from __future__ import annotations

import math

import numpy as np

import oracle as O
from paper_1102_5202_gb300 import hzn
from paper_1102_5202_gb300 import workloads as W

# FP64 tolerances of the benchmark statement: relative L1 per field
TOL_ONE_STEP = 1e-10
TOL_END = 1e-8

# End-time bar where the workload itself amplifies rounding: the GPU result may differ from the
# oracle's by at most this factor times the oracle's own spread, the largest relative L1 per
# field between the oracle run and the oracle runs from one-ulp perturbations of its input (the
# same steps).  A discrete decision (the atmosphere threshold, a limiter or monotonicity switch)
# that an ulp flips turns rounding into an O(1) change of one cell, which then spreads; which
# perturbation flips which decision first is chance, so several perturbations are taken.
SPREAD_FACTOR = 10.0


def oracle_setup(P):
    grid = O.make_grid(P.n, P.dx, P.bc)
    opts = O.make_opts(P.gamma, cleaning=P.cleaning, ch=P.ch, kappa=P.kappa, rho_floor=P.rho_floor,
                       p_floor=P.p_floor, atm_K=P.atm_K, rho_atm=P.rho_atm, recon=P.recon)
    return grid, opts


def oracle_run(P, nsteps=1, dt=None, t_end=None, cfl=None):
    grid, opts = oracle_setup(P)
    U = O.grid_prim2cons(grid, opts, P.metric, P.prim)
    if t_end is not None:
        prim, cons, steps, t, nf = O.evolve(grid, opts, P.metric, P.prim, U, t_end, cfl)
        return prim, cons, dict(steps=steps, t=t, fails=nf)
    prim, cons = P.prim, U
    fails = 0
    for _ in range(nsteps):
        prim, cons, nf = O.step(grid, opts, P.metric, prim, cons, dt)
        fails += nf
    return prim, cons, dict(steps=nsteps, t=nsteps * dt, fails=fails)


def gpu_solver(P, **kw):
    return hzn.Solver.for_problem(P, **kw)


def gpu_run(P, nsteps=1, dt=None, t_end=None, cfl=None, solver=None):
    import torch

    s = solver or gpu_solver(P)
    if t_end is not None:
        s.evolve(t_end, cfl)
    else:
        for _ in range(nsteps):
            s.step(dt)
    prim = s.primitives().cpu().numpy()
    cons = s.conserved().cpu().numpy()
    st = s.stats()
    torch.cuda.synchronize()
    return prim, cons, dict(steps=st.steps, t=st.t, fails=st.c2p_failures, maxit=st.c2p_max_iters,
                            max_speed=st.max_speed)


# Components of one vector share one scale: (rho), (p | T_t), (u~^i | T_i), (B^i), (psi).
FIELD_GROUPS = ((0,), (1,), (2, 3, 4), (5, 6, 7), (8,))


def rel_l1(a, b):
    """Per-field relative L1 error: sum|a_f - b_f| / sum |b_G| where |b_G| is the Euclidean
    magnitude of the vector the field belongs to (the field itself for a scalar); absolute
    sum|a - b| where the reference is identically 0."""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    num = np.abs(a - b).sum(axis=1)
    den = np.zeros(a.shape[0])
    for grp in FIELD_GROUPS:
        if grp[0] >= a.shape[0]:
            continue
        mag = np.sqrt((b[list(grp)] ** 2).sum(axis=0)).sum()
        for f in grp:
            den[f] = mag
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def assert_parity(gpu, orc, tol, fields=None, what=""):
    r = rel_l1(gpu, orc)
    idx = range(gpu.shape[0]) if fields is None else fields
    bad = [(W.PRIM_FIELDS[f] if gpu.shape[0] == 9 else f, float(r[f])) for f in idx if not (r[f] <= tol)]
    assert not bad, f"{what} relative L1 above {tol}: {bad}"
    return r


def tile_tube(P1, axis: int, other: int = 3) -> W.Problem:
    """Embed a 1-D tube along x into a grid where the tube runs along ``axis`` and the other
    active axes are periodic with ``other`` identical cells (x stays active)."""
    n1 = P1.n[0]
    prim1 = P1.prim[:, 0, 0, :]  # (9, n1)
    perm = [(0, 1, 2), (1, 2, 0), (2, 0, 1)][axis]
    q = prim1.copy()
    for k in range(3):
        q[2 + perm[k]] = prim1[2 + k]
        q[5 + perm[k]] = prim1[5 + k]
    if axis == 0:
        n = (n1, other, 1)
    elif axis == 1:
        n = (other, n1, 1)
    else:
        n = (other, other, n1)
    prim = np.empty((9, n[2], n[1], n[0]))
    for f in range(9):
        if axis == 0:
            prim[f] = q[f][None, None, :]
        elif axis == 1:
            prim[f] = q[f][None, :, None]
        else:
            prim[f] = q[f][:, None, None]
    dx = [P1.dx[0] * 1.0] * 3
    bc = [1, 1, 1]
    bc[axis] = P1.bc[0]
    return W.Problem(P1.name + f"_ax{axis}", n, tuple(dx), (0.0, 0.0, 0.0), tuple(bc), P1.gamma,
                     np.ascontiguousarray(prim), W.minkowski_metric(n), t_end=P1.t_end, cfl=P1.cfl,
                     cleaning=P1.cleaning, ch=P1.ch, kappa=P1.kappa)


def general_metric(X, Y, Z):
    """A smooth periodic general static metric: lapse, shift and non-diagonal gamma_ij."""
    m = np.zeros((10,) + X.shape)
    m[0] = 0.85 + 0.1 * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y)
    m[1] = 0.05 * np.sin(2 * math.pi * Y)
    m[2] = -0.03 * np.cos(2 * math.pi * Z)
    m[3] = 0.02 * np.sin(2 * math.pi * X)
    psi4 = 1.2 + 0.1 * np.cos(2 * math.pi * Z) * np.sin(2 * math.pi * X)
    m[4] = psi4
    m[7] = psi4 * 1.05
    m[9] = psi4 * 0.95
    m[5] = 0.02 * np.cos(2 * math.pi * Z)
    m[6] = -0.015 * np.sin(2 * math.pi * Y)
    m[8] = 0.01 * np.cos(2 * math.pi * X)
    return m


def perturbed(P, kind: str, seed: int = 5):
    """P with its primitive input moved by one ulp: 'rho' up, 'p' down, or 'all' (every
    field, in a seeded random direction)."""
    import dataclasses

    prim = P.prim.copy()
    if kind == "rho":
        prim[0] = np.nextafter(prim[0], np.inf)
    elif kind == "p":
        prim[1] = np.nextafter(prim[1], -np.inf)
    elif kind == "all":
        rng = np.random.Generator(np.random.PCG64(seed))
        prim = np.nextafter(prim, rng.choice([-np.inf, np.inf], size=prim.shape))
    else:
        raise ValueError(kind)
    return dataclasses.replace(P, prim=prim)


def oracle_replay(P, dts):
    """The oracle from P's input over the given time steps: (prim, cons)."""
    grid, opts = oracle_setup(P)
    U = O.grid_prim2cons(grid, opts, P.metric, P.prim)
    prim = P.prim
    for dt in dts:
        prim, U, _ = O.step(grid, opts, P.metric, prim, U, dt)
    return prim, U


def integral_diff(a, b):
    """|sum a_f - sum b_f| / sum |b_f| per conserved field over the grid."""
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return np.abs(a.sum(axis=1) - b.sum(axis=1)) / np.maximum(np.abs(b).sum(axis=1), 1e-300)


def oracle_spread(P, ref_prim, run, kinds=("rho", "p", "all")):
    """The oracle's own spread on this case: the largest relative L1 per field between
    ref_prim (the oracle run from P) and run(Q) for the one-ulp perturbations Q of P."""
    spread = np.zeros(ref_prim.shape[0])
    for kind in kinds:
        spread = np.maximum(spread, rel_l1(run(perturbed(P, kind)), ref_prim))
    return spread


def assert_within_spread(gpu, orc, spread, what="", fields=None):
    """GPU vs oracle per field within max(TOL_END, SPREAD_FACTOR x the oracle's spread)."""
    r = rel_l1(gpu, orc)
    bar = np.maximum(TOL_END, SPREAD_FACTOR * spread)
    idx = range(gpu.shape[0]) if fields is None else fields
    bad = [(W.PRIM_FIELDS[f], float(r[f]), float(bar[f])) for f in idx if not (r[f] <= bar[f])]
    assert not bad, f"{what}: relative L1 above the spread bar (field, got, bar): {bad}"
    return r, bar
