"""Checks of the double-word (pair-of-FP32) operations of the HZ_FP64_DW path against exact
decimal arithmetic, shared by the GPU test (the library's hz_dw_selftest) and the CPU test (a
host build of the same headers)."""
from __future__ import annotations

import decimal

import numpy as np

NRESULTS = 9  # x, y, x + y, x - y, x * y, x / y, sqrt|x|, 1/sqrt|x|, half MC slope


def pair_inputs(seed: int = 2026, n: int = 600):
    """(a, b, m): m general, cancelling, equal / opposite and special pairs, then values for the
    split alone over the FP32 exponent range (b = 1 there)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mag = lambda k, lo, hi: 10.0 ** rng.uniform(lo, hi, k) * rng.choice([-1.0, 1.0], k)
    a = np.concatenate([mag(n, -12, 12), mag(n, -6, 6), mag(n, -12, 12), [0.0, 1.0, -2.5, 3.0]])
    b = np.concatenate([mag(n, -12, 12), -a[n:2 * n] * (1 + mag(n, -15, -3)),
                        a[2 * n:3 * n].copy(), [2.0, 0.0, -2.5, 3.0]])
    b[2 * n:3 * n:2] *= -1.0  # exact equal and exactly opposite pairs
    wide = mag(400, -30, 37)  # below ~1e-31 the trailing float is subnormal (fewer bits)
    m = len(a)
    return np.concatenate([a, wide]), np.concatenate([b, np.ones_like(wide)]), m


def check_pair_results(a, out, m):
    """out: (NRESULTS, 2, len(a)) of (hi, lo).  Bounds, with u = 2^-24: split within 2^-47
    relative; sum and difference within 4u^2(|x| + |y|) (through cancellation); product 6u^2,
    quotient and square root 16u^2, inverse square root 32u^2 relative; the half MC slope within
    4u^2(|x| + |y|) of the exact limited slope of the pair inputs; every result normalised
    (|lo| <= ulp(hi))."""
    D = decimal.Decimal
    decimal.getcontext().prec = 100
    u2 = D(2) ** -48

    def val(q, i):
        hi, lo = out[q, 0, i], out[q, 1, i]
        assert (hi == 0.0 and lo == 0.0) or abs(lo) <= abs(hi) * 2.0 ** -23, (q, i, hi, lo)
        return D(float(hi)) + D(float(lo))

    for i in range(len(a)):
        X = val(0, i)
        src = D(float(a[i]))
        assert abs(X - src) <= D(2) ** -47 * abs(src), ("split", i)
        if i >= m:
            continue
        Y = val(1, i)
        s = abs(X) + abs(Y)
        assert abs(val(2, i) - (X + Y)) <= 4 * u2 * s, ("add", i)
        assert abs(val(3, i) - (X - Y)) <= 4 * u2 * s, ("sub", i)
        assert abs(val(4, i) - X * Y) <= 6 * u2 * abs(X * Y), ("mul", i)
        if Y != 0:
            assert abs(val(5, i) - X / Y) <= 16 * u2 * abs(X / Y), ("div", i)
        r = abs(X).sqrt()
        assert abs(val(6, i) - r) <= 16 * u2 * r, ("sqrt", i)
        if X != 0:
            assert abs(val(7, i) - 1 / r) <= 32 * u2 / r, ("rsqrt", i)
        same = (X > 0 and Y > 0) or (X < 0 and Y < 0)
        want = D(0)
        if same:
            want = min(abs(X), abs(Y), abs(X + Y) / 4)
            want = want if Y > 0 else -want
        assert abs(val(8, i) - want) <= 4 * u2 * s, ("mc", i)
