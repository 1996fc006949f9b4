"""CPU check of the screening's per-query dot threshold (no GPU). The emission pass keeps a
(row, query) pair for its exact interval test when dot >= L, L = rd(rd(xn_min - R+) / 2), where
R = ru(ru(thr + M_max) - |q|^2) and R+ is the next fp32 value above R; that must keep every
pair that the range test rd(xn_min - 2 dot) <= R keeps. Checked with exact rational arithmetic
for the directed roundings, on random values and on dots placed at and around the boundary."""
from fractions import Fraction

import numpy as np

F32 = np.float32


def rd(x: Fraction) -> F32:
    """Largest fp32 value <= x (x finite, in range)."""
    f = F32(float(x))
    while Fraction(float(f)) > x:
        f = np.nextafter(f, F32(-np.inf))
    while Fraction(float(np.nextafter(f, F32(np.inf)))) <= x:
        f = np.nextafter(f, F32(np.inf))
    return f


def next_up(r: F32) -> F32:
    return np.nextafter(r, F32(np.inf))


def test_threshold_keeps_every_pair_the_range_test_keeps():
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(4000):
        xn_min = F32(rng.uniform(200.0, 300.0))
        R = F32(rng.uniform(-300.0, 300.0))
        L = rd(Fraction(float(rd(Fraction(float(xn_min)) - Fraction(float(next_up(R)))))) / 2)
        # dots around the boundary (xn_min - R) / 2 and around L itself
        centre = (float(xn_min) - float(R)) / 2
        dots = [F32(centre + d) for d in (-1e-3, -1e-5, 0.0, 1e-5, 1e-3)]
        f = F32(L)
        for _ in range(3):
            dots += [f]
            f = np.nextafter(f, F32(-np.inf))
        dots += [np.nextafter(F32(L), F32(np.inf))]
        for dot in dots:
            kept_by_range = rd(Fraction(float(xn_min)) - 2 * Fraction(float(dot))) <= R
            if kept_by_range:
                assert dot >= L, (xn_min, R, dot, L)
                checked += 1
        # and it is not looser than a few fp32 steps: a dot clearly below the boundary fails
        assert not (F32(centre - 1e-3) >= L)
    assert checked > 1000
