"""Planted segments that stress exact PAA (Sec. 2.2: PAA = mean of each segment).

The PAA of a segment is the exact real sum of its s fp32 values, rounded once to FP64 and
divided by s. A summation that loses a low bit anywhere shows up on these inputs:

* ``wide_span`` segments: half the values near 2 (the running sum crosses a power of two,
  so its ulp doubles) and half near 2^-15 with a low bit set, so every addition leaves a
  rounding error that must be carried exactly (exponent span 15);
* ``gate`` segments: random full-significand values whose exponents span exactly a given
  number of binades, for spans on both sides of any exponent-span rule an implementation uses;
* ``below_breakpoint`` segments: values whose exact sum is the largest multiple of their
  common quantum below s * beta_j. Their exact PAA lies less than 2^-38 / s below the
  breakpoint, so a sum that errs upward by more than that crosses it and changes the iSAX
  symbol (and, for j = 192, plane 1 of the key).

Everything here is exact host arithmetic (``fractions.Fraction``); nothing is taken from the
library under test.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

F32 = np.float32
A_NEAR_TWO = F32(1.9999999)
B_LOW_BIT = F32(2.0 ** -15 + 2.0 ** -18 - 2.0 ** -38)


def wide_span(s: int, rng: np.random.Generator, variant: int) -> np.ndarray:
    """s values: s/2 copies of ~2 then s/2 copies of ~2^-15 (variant 0), shuffled (1),
    random signs (2), reversed (3)."""
    v = np.concatenate([np.full(s // 2, A_NEAR_TWO), np.full(s - s // 2, B_LOW_BIT)]).astype(F32)
    if variant == 1:
        v = v[rng.permutation(s)]
    elif variant == 2:
        v = v * np.where(rng.random(s) < 0.5, F32(-1), F32(1)).astype(F32)
    elif variant == 3:
        v = v[::-1].copy()
    return v


def gate(s: int, span: int, rng: np.random.Generator) -> np.ndarray:
    """s values with full random significands whose binary exponents cover exactly [e0-span, e0]
    (the largest first, so the running sum is large when the small values arrive)."""
    e0 = int(rng.integers(-2, 3))
    exps = e0 - rng.integers(0, span + 1, size=s)
    exps[0] = e0
    exps[-1] = e0 - span
    mant = 1.0 + rng.integers(0, 1 << 23, size=s).astype(np.float64) / (1 << 23)
    sign = np.where(rng.random(s) < 0.25, -1.0, 1.0)
    return (sign * np.ldexp(mant, exps)).astype(F32)


def _exact_sum(vals) -> Fraction:
    return sum((Fraction(float(v)) for v in vals), Fraction(0))


def below_breakpoint(beta: float, s: int, order: str = "plain", seed: int = 0) -> np.ndarray:
    """s values (s >= 16) whose exact sum is the largest one reachable below s * beta with the
    last value in [2^-15, 2^-14): s/2 values ~2 push the sum across a binade, s/4 values ~2^-15
    add a rounding error each, the rest (~-(2 - beta)) bring the sum down to s * beta, and the
    last value closes the gap to within its quantum 2^-38. ``order`` = "plain", "reversed" or
    "shuffled" (the exact sum does not depend on the order)."""
    assert s >= 16
    n_a, n_b = s // 2, s // 4
    n_c = s - n_a - n_b - 2
    head = [A_NEAR_TWO] * n_a + [B_LOW_BIT] * n_b
    target = Fraction(float(beta)) * s
    c = F32(float((target - _exact_sum(head)) / (n_c + 1)) - 1.5 * 2.0 ** -15 / (n_c + 1))
    base = None
    for step in range(0, 1 << 16):
        for sgn in (1, -1):
            c1 = F32(float(c) + sgn * step * float(np.spacing(c)))
            trial = head + [c] * n_c + [c1]
            rest = target - _exact_sum(trial)
            if Fraction(2) ** -15 <= rest < Fraction(2) ** -14:
                base = trial
                break
        if base is not None:
            break
    assert base is not None
    rest = target - _exact_sum(base)
    d = F32(float(rest))
    while Fraction(float(d)) >= rest:
        d = np.nextafter(d, F32(-np.inf), dtype=F32)
    while Fraction(float(np.nextafter(d, F32(np.inf), dtype=F32))) < rest:
        d = np.nextafter(d, F32(np.inf), dtype=F32)
    vals = np.array(base + [d], dtype=F32)
    if order == "reversed":
        vals = vals[::-1].copy()
    elif order == "shuffled":
        vals = vals[np.random.default_rng(seed).permutation(s)]
    return vals


def exact_mean(vals) -> Fraction:
    return _exact_sum(vals) / len(vals)
