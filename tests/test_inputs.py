"""Seeded inputs that carry physics of their own (CPU): the toroidal-field blob of §5.2 and the
gradient workloads."""
import math

import numpy as np

from paper_1102_5202_gb300 import workloads as W


def _centred_divergence(P):
    """Max over interior cells of |d_i (sqrt(gamma) B^i)| dx / max |sqrt(gamma) B|, centred."""
    met = P.metric[:, 1:-1, 1:-1, 1:-1]
    sqrtg = met[4] ** 1.5  # conformally flat: gamma_ij = psi^4 delta_ij
    F = [sqrtg * P.prim[5 + d] for d in range(3)]
    div = (F[0][1:-1, 1:-1, 2:] - F[0][1:-1, 1:-1, :-2] + F[1][1:-1, 2:, 1:-1] - F[1][1:-1, :-2, 1:-1] +
           F[2][2:, 1:-1, 1:-1] - F[2][:-2, 1:-1, 1:-1]) / 2.0
    return np.abs(div).max() / max(np.abs(f).max() for f in F)


def test_toroidal_field_is_divergence_free_to_second_order():
    e = [_centred_divergence(W.blob3d(n, field="toroidal")) for n in (32, 64)]
    assert e[1] < e[0] / 3.0, e  # O(dx^2) truncation of the centred difference


def test_toroidal_field_strength_and_shape():
    # continuum maximum at varpi = varpi0, z = 0: B0 / e = 2.6e15 G in code units
    peak = W.toroidal_profile(np.array([W.TOROIDAL_VARPI0]), np.array([0.0]), np.array([0.0]))[0]
    assert abs(peak - 1.0 / math.e) < 1e-15
    P = W.blob3d(48, field="toroidal")
    met = P.metric[:, 1:-1, 1:-1, 1:-1]
    bn = np.sqrt(met[4] * met[0] ** 2 * (P.prim[5] ** 2 + P.prim[6] ** 2 + P.prim[7] ** 2))
    target = W.TOROIDAL_B_GAUSS / W.GAUSS_PER_CODE_UNIT
    assert target * 0.8 < bn.max() <= target * (1 + 1e-12)
    assert np.all(P.prim[7] == 0.0)
    # toroidal: B is perpendicular to the cylindrical radius
    n = P.n[0]
    c = P.x0[0] + (np.arange(n) + 0.5) * P.dx[0]
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    assert np.abs(X * P.prim[5] + Y * P.prim[6]).max() < 1e-12 * np.abs(P.prim[5]).max() * 20
    # the rest of the state is the poloidal blob's
    Q = W.blob3d(48)
    assert np.array_equal(P.prim[:5], Q.prim[:5]) and np.array_equal(P.metric, Q.metric)


def test_gradient_workload_fixed_step_is_the_multi_axis_light_speed_bound():
    T = W.adjoint_tube(100)
    B = W.blast2d(64)
    assert W.fixed_dt(T) == T.cfl * T.dx[0]
    assert abs(W.fixed_dt(B) - 0.5 * B.cfl * B.dx[0]) < 1e-18
