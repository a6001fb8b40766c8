"""Exact solution of the special-relativistic Riemann problem of an ideal gas with zero
tangential velocity (the unmagnetised shock tubes of §5.1).  Test infrastructure: it pins the
oracle to a closed-form solution.

Waves: a rarefaction follows the isentrope p = K rho^Gamma along which the Riemann invariant
artanh(v) +- I(rho), I = integral of c_s / rho d rho, is constant (integrated numerically
here); a shock follows the Taub adiabat [h^2] = (h_b/rho_b + h_a/rho_a)[p] with mass flux
j^2 = -[p] / [h/rho] and the shock and post-shock velocities of the standard jump conditions.
The star pressure is the root of v_left*(p) = v_right*(p).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize


class IdealGas:
    def __init__(self, gamma: float):
        self.g = gamma

    def h(self, rho, p):
        return 1.0 + self.g / (self.g - 1.0) * p / rho

    def cs(self, rho, p):
        return math.sqrt(self.g * p / (rho * self.h(rho, p)))

    def rho_from_hp(self, h, p):
        return self.g * p / ((self.g - 1.0) * (h - 1.0))


def _rarefaction_I(eos: IdealGas, rho_a, p_a, rho):
    K = p_a / rho_a ** eos.g
    f = lambda r: eos.cs(r, K * r ** eos.g) / r
    val, _ = integrate.quad(f, rho_a, rho, epsabs=1e-14, epsrel=1e-13, limit=200)
    return val


def rarefaction_state(eos, rho_a, p_a, v_a, p, sign):
    """State behind a rarefaction reached at pressure p. sign=-1 left wave, +1 right wave."""
    K = p_a / rho_a ** eos.g
    rho = (p / K) ** (1.0 / eos.g)
    I = _rarefaction_I(eos, rho_a, p_a, rho)
    v = math.tanh(math.atanh(v_a) + sign * I)
    return rho, v


def shock_state(eos, rho_a, p_a, v_a, p_b, sign):
    """Post-shock (rho_b, v_b, V_s) for a shock into state a.  sign=-1 left, +1 right."""
    g = eos.g
    h_a = eos.h(rho_a, p_a)
    dp = p_b - p_a
    c = (g - 1.0) * dp / (g * p_b)
    # h_b^2 (1 - c) + h_b c - h_a^2 - h_a dp / rho_a = 0
    A, B, C = 1.0 - c, c, -(h_a * h_a + h_a * dp / rho_a)
    h_b = (-B + math.sqrt(B * B - 4.0 * A * C)) / (2.0 * A)
    rho_b = eos.rho_from_hp(h_b, p_b)
    j2 = -dp / (h_b / rho_b - h_a / rho_a)
    j = sign * math.sqrt(j2)
    W_a = 1.0 / math.sqrt(1.0 - v_a * v_a)
    a2 = rho_a * rho_a * W_a * W_a
    Vs = (a2 * v_a + j * math.sqrt(j2 + a2 * (1.0 - v_a * v_a))) / (a2 + j2)
    Ws = 1.0 / math.sqrt(1.0 - Vs * Vs)
    v_b = (h_a * W_a * v_a + Ws * dp / j) / (h_a * W_a + dp * (Ws * v_a / j + 1.0 / (rho_a * W_a)))
    return rho_b, v_b, Vs


class RiemannSolution:
    def __init__(self, gamma, left, right):
        """left/right = (rho, p, v)."""
        self.eos = IdealGas(gamma)
        self.L, self.R = left, right
        rl, pl, vl = left
        rr, pr, vr = right

        def vstar(p, side):
            rho_a, p_a, v_a = left if side < 0 else right
            if p > p_a:
                return shock_state(self.eos, rho_a, p_a, v_a, p, side)[1]
            return rarefaction_state(self.eos, rho_a, p_a, v_a, p, side)[1]

        fn = lambda p: vstar(p, -1) - vstar(p, +1)
        lo, hi = min(pl, pr) * 1e-6, max(pl, pr) * 1e3
        self.pstar = optimize.brentq(fn, lo, hi, xtol=1e-15, rtol=1e-14, maxiter=500)
        self.vstar = vstar(self.pstar, -1)
        self.waves = []
        for side in (-1, +1):
            rho_a, p_a, v_a = left if side < 0 else right
            if self.pstar > p_a:
                rho_s, v_s, Vs = shock_state(self.eos, rho_a, p_a, v_a, self.pstar, side)
                self.waves.append(("shock", rho_s, Vs))
            else:
                rho_s, v_s = rarefaction_state(self.eos, rho_a, p_a, v_a, self.pstar, side)
                self.waves.append(("raref", rho_s, None))

    def _lam(self, rho, p, v, side):
        c = self.eos.cs(rho, p)
        return (v + side * c) / (1.0 + side * v * c)

    def _fan(self, xi, side):
        """State inside a rarefaction fan at similarity coordinate xi."""
        rho_a, p_a, v_a = self.L if side < 0 else self.R
        K = p_a / rho_a ** self.eos.g

        def g(rho):
            p = K * rho ** self.eos.g
            I = _rarefaction_I(self.eos, rho_a, p_a, rho)
            v = math.tanh(math.atanh(v_a) + side * I)
            return self._lam(rho, p, v, side) - xi

        rho_star = self.waves[0 if side < 0 else 1][1]
        lo, hi = min(rho_star, rho_a), max(rho_star, rho_a)
        rho = optimize.brentq(g, lo, hi, xtol=1e-15, rtol=1e-14, maxiter=500)
        p = K * rho ** self.eos.g
        I = _rarefaction_I(self.eos, rho_a, p_a, rho)
        return rho, p, math.tanh(math.atanh(v_a) + side * I)

    def sample(self, xi: float):
        """(rho, p, v) at similarity coordinate xi = (x - x_c) / t."""
        rl, pl, vl = self.L
        rr, pr, vr = self.R
        # left wave
        kind, rho_sl, Vs = self.waves[0]
        if kind == "shock":
            if xi < Vs:
                return rl, pl, vl
        else:
            head = self._lam(rl, pl, vl, -1)
            tail = self._lam(rho_sl, self.pstar, self.vstar, -1)
            if xi < head:
                return rl, pl, vl
            if xi < tail:
                return self._fan(xi, -1)
        if xi < self.vstar:
            return rho_sl, self.pstar, self.vstar
        kind, rho_sr, Vs = self.waves[1]
        if kind == "shock":
            if xi < Vs:
                return rho_sr, self.pstar, self.vstar
            return rr, pr, vr
        tail = self._lam(rho_sr, self.pstar, self.vstar, +1)
        head = self._lam(rr, pr, vr, +1)
        if xi < tail:
            return rho_sr, self.pstar, self.vstar
        if xi < head:
            return self._fan(xi, +1)
        return rr, pr, vr

    def cell_average(self, x_lo, x_hi, x_c, t, sub=16):
        """Cell-averaged (rho, p, v) by midpoint quadrature over ``sub`` points."""
        xs = x_lo + (np.arange(sub) + 0.5) * (x_hi - x_lo) / sub
        vals = np.array([self.sample((x - x_c) / t) for x in xs])
        return vals.mean(axis=0)
