"""Pins of the oracle's PPM reconstruction (§3.2) and of the full update with it.

The reconstruction is checked against what PPM fixes: face values exact for cell averages of a
cubic where no limiter acts, no parabola with an extremum inside its cell, a flat profile in a
cell at a local extremum, and the MC states unchanged.  The update is checked by conservation
in a periodic box, convergence to the exact Sod solution, and a smooth wave converging faster
than with MC."""
import math

import numpy as np

from exact_riemann import RiemannSolution
from parity import oracle_setup
from paper_1102_5202_gb300 import workloads as W
import oracle as O

PPM = O.RECON_PPM


def _cell_averages(F, edges):
    return (F(edges[1:]) - F(edges[:-1])) / np.diff(edges)


def test_ppm_faces_exact_for_cubic_averages():
    # f = 1 + x + 0.3 x^2 + 0.05 x^3 is monotone with small curvature on [0, 1]: the MC slopes
    # are the central ones and no monotonicity constraint acts, so the interface values of
    # cell averages reproduce f at the faces exactly (the interpolating parabola construction
    # is exact for cubics).
    f = lambda x: 1 + x + 0.3 * x ** 2 + 0.05 * x ** 3
    F = lambda x: x + 0.5 * x ** 2 + 0.1 * x ** 3 + 0.0125 * x ** 4
    n = 24
    edges = np.linspace(0.0, 1.0, n + 1)
    q = _cell_averages(F, edges)
    left, right = O.reconstruct_1d(PPM, q)
    c = np.arange(3, n - 2)
    exact = f(edges[c])
    assert np.abs(left[c] - exact).max() < 1e-13
    assert np.abs(right[c] - exact).max() < 1e-13
    # MC on the same data is only second order: it does not reproduce the face values
    lm, _ = O.reconstruct_1d(O.RECON_MC, q)
    assert np.abs(lm[c] - exact).max() > 1e-6


def test_ppm_parabolas_have_no_interior_extremum():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = 40
        q = np.cumsum(rng.standard_normal(n)) if trial % 2 else rng.standard_normal(n)
        left, right = O.reconstruct_1d(PPM, q)
        # cell c has aL = right[c] (its left face) and aR = left[c + 1]
        for c in range(3, n - 3):
            aL, aR, a = right[c], left[c + 1], q[c]
            if aL == a and aR == a:
                continue
            d = aR - aL
            m6 = 6.0 * (a - 0.5 * (aL + aR))
            assert abs(m6) <= abs(d) * (1 + 1e-12) + 1e-15, (trial, c, aL, a, aR)
            # and the cell value lies between its edge values
            assert min(aL, aR) - 1e-15 <= a <= max(aL, aR) + 1e-15


def test_ppm_flattens_a_local_extremum():
    q = np.array([0.0, 1.0, 2.0, 3.0, 4.5, 3.0, 2.0, 1.0, 0.0, -0.5, -0.7])
    left, right = O.reconstruct_1d(PPM, q)
    peak = 4
    assert right[peak] == q[peak] and left[peak + 1] == q[peak]


def test_ppm_face_values_bounded_by_neighbours_for_steps():
    rng = np.random.default_rng(11)
    q = np.cumsum(np.where(rng.random(50) < 0.3, rng.random(50) * 5.0, 0.0))  # monotone steps
    left, right = O.reconstruct_1d(PPM, q)
    for c in range(3, len(q) - 2):
        lo, hi = min(q[c - 1], q[c]), max(q[c - 1], q[c])
        assert lo - 1e-12 <= left[c] <= hi + 1e-12
        assert lo - 1e-12 <= right[c] <= hi + 1e-12


def _ppm(P):
    P.recon = PPM
    return P


def test_ppm_conservation_periodic():
    P = _ppm(W.smooth_periodic((12, 10, 8), seed=7, amp=0.2, magnetised=True))
    grid, opts = oracle_setup(P)
    U0 = O.grid_prim2cons(grid, opts, P.metric, P.prim)
    dt = 0.4 / O.max_speed(grid, opts, P.metric, P.prim)
    prim, U = P.prim, U0
    for _ in range(4):
        prim, U, nf = O.step(grid, opts, P.metric, prim, U, dt)
        assert nf == 0
    tot0 = U0.reshape(9, -1).sum(axis=1)
    tot = U.reshape(9, -1).sum(axis=1)
    scale = np.abs(U0).reshape(9, -1).sum(axis=1) + 1e-300
    assert np.all(np.abs(tot - tot0)[:8] <= 1e-13 * scale[:8])


def _sod_l1(n, recon):
    P = W.sod(n)
    P.recon = recon
    grid, opts = oracle_setup(P)
    U = O.grid_prim2cons(grid, opts, P.metric, P.prim)
    prim, _, _, t, nf = O.evolve(grid, opts, P.metric, P.prim, U, 0.4, 0.5)
    assert nf == 0
    sol = RiemannSolution(P.gamma, (1.0, 1.0, 0.0), (0.125, 0.1, 0.0))
    xs = P.x0[0] + np.arange(n) * P.dx[0]
    ex = np.array([sol.cell_average(x, x + P.dx[0], 0.0, t) for x in xs])
    return np.abs(prim[0].ravel() - ex[:, 0]).mean()


def test_ppm_sod_converges_to_exact_solution():
    e100, e400 = _sod_l1(100, PPM), _sod_l1(400, PPM)
    assert e400 < e100 / 2.5
    assert e400 < 2e-3
    assert e400 < _sod_l1(400, O.RECON_MC)  # sharper than MC on the same grid


def _entropy_l1(n, recon):
    dx = 1.0 / n
    xs = (np.arange(n) + 0.5) * dx
    v = 0.5
    prim = np.zeros((9, 1, 1, n))
    prim[0] = 1.0 + 0.2 * (np.cos(2 * math.pi * (xs - dx / 2)) - np.cos(2 * math.pi * (xs + dx / 2))) / (2 * math.pi * dx)
    prim[1] = 1.0
    prim[2] = v / math.sqrt(1 - v * v)
    P = W.Problem("ent", (n, 1, 1), (dx, 1.0, 1.0), (0.0, 0.0, 0.0), (1, 1, 1), 5.0 / 3.0,
                  prim, W.minkowski_metric((n, 1, 1)))
    P.recon = recon
    grid, opts = oracle_setup(P)
    U = O.grid_prim2cons(grid, opts, P.metric, P.prim)
    out, _, _, t, _ = O.evolve(grid, opts, P.metric, P.prim, U, 0.4, 0.4)
    ex = 1.0 + 0.2 * (np.cos(2 * math.pi * (xs - dx / 2 - v * t)) - np.cos(2 * math.pi * (xs + dx / 2 - v * t))) / (2 * math.pi * dx)
    return np.abs(out[0].ravel() - ex).mean()


def test_ppm_smooth_wave_converges_faster_than_mc():
    e = [_entropy_l1(n, PPM) for n in (64, 128, 256)]
    order = math.log2(e[1] / e[2])
    assert order > 2.15, e
    assert e[2] < _entropy_l1(256, O.RECON_MC)
