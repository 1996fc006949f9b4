"""CPU check of the error bound behind the build's fp32 symbol decision (no GPU).

The build decides a segment's symbol from the fp32 sum S of its s values when the interval
[P - E, P + E] around P = S / s, E = M * (s - 1) * 2^-24 * (1 + 2^-15) + 2^-148 (M = largest
magnitude), holds no breakpoint; the exact PAA p = RN64(exact sum) / s must then have the same
symbol. This test emulates that decision in numpy fp32 with outward-rounded interval ends (each
end moved one fp32 step outward, which is at least as wide as directed rounding) and checks,
on random segments and on segments built to sit at or next to breakpoints, that every decided
symbol equals the oracle's symbol of the exact PAA, and that the undecided lanes are rare on
random walks."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import isax

F32 = np.float32


def fp32_sum(vals):
    acc = F32(0.0)
    for v in vals:
        acc = F32(acc + F32(v))
    return acc


def decide(vals, s, beta_lo, beta_hi, card):
    """The decided symbol, or None when a breakpoint lies within the bound."""
    L = s.bit_length() - 1
    M = F32(np.max(np.abs(vals)))
    S = fp32_sum(vals)
    P = F32(S * F32(2.0 ** -L))
    cE = np.nextafter(F32((s - 1) * 2.0 ** -24 * (1 + 2.0 ** -15)), F32(np.inf))
    E = np.nextafter(F32(np.nextafter(F32(M * cE), F32(np.inf)) + F32(2.0 ** -148)), F32(np.inf))
    lo = np.nextafter(F32(P - E), F32(-np.inf))
    hi = np.nextafter(F32(P + E), F32(np.inf))
    s0 = int(np.searchsorted(beta_lo, P, side="right"))  # candidate: breakpoints <= P
    s0 = min(s0, card - 1)
    ok_lo = s0 == 0 or beta_hi[s0 - 1] <= lo
    ok_hi = s0 == card - 1 or beta_lo[s0] > hi
    return s0 if (ok_lo and ok_hi) else None


def brackets(card):
    beta = isax.breakpoints(card)
    lo = np.array([np.nextafter(F32(b), F32(-np.inf)) if float(F32(b)) > b else F32(b) for b in beta], F32)
    hi = np.array([np.nextafter(F32(b), F32(np.inf)) if float(F32(b)) < b else F32(b) for b in beta], F32)
    assert np.all(lo.astype(np.float64) <= beta) and np.all(hi.astype(np.float64) >= beta)
    return beta, lo, hi


def exact_symbol(vals, s, card):
    exact = sum(Fraction(float(v)) for v in vals)
    p = float(exact) / s                       # RN64 of the exact sum, then an exact division
    return int(isax.symbols(np.array([p]), card)[0])


@pytest.mark.parametrize("s", [4, 8, 16])
def test_decided_symbols_are_exact_on_random_walk_segments(s):
    import synth
    card = 256
    _, blo, bhi = brackets(card)
    x = synth.random_walk(400, 16 * s, seed=90 + s)
    undecided = 0
    total = 0
    for row in x:
        for i in range(16):
            seg = row[i * s:(i + 1) * s]
            got = decide(seg, s, blo, bhi, card)
            total += 1
            if got is None:
                undecided += 1
                continue
            assert got == exact_symbol(seg, s, card)
    assert undecided <= total // 200          # well under 0.5% of the lanes take the exact sum


@pytest.mark.parametrize("s", [4, 8, 16])
def test_segments_at_and_next_to_breakpoints(s):
    """Every value equal to the fp32 value nearest a breakpoint, or one step above or below it:
    the mean is that value, within one step of the breakpoint; a decided symbol must be exact,
    and a mean equal to a breakpoint must never be decided (it needs the upper-region tie rule)."""
    card = 256
    beta, blo, bhi = brackets(card)
    for j in range(0, 255, 3):
        c = F32(beta[j])
        for v in (c, np.nextafter(c, F32(np.inf)), np.nextafter(c, F32(-np.inf))):
            seg = np.full(s, v, F32)
            got = decide(seg, s, blo, bhi, card)
            if got is not None:
                assert got == exact_symbol(seg, s, card)
            if float(v) == beta[j]:
                assert got is None


def test_planted_sums_just_below_breakpoints():
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    import planted
    card = 256
    beta, blo, bhi = brackets(card)
    for j in (64, 128, 160, 192):
        for order in ("plain", "reversed", "shuffled"):
            seg = planted.below_breakpoint(beta[j - 1], 16, order, seed=j)
            got = decide(seg, 16, blo, bhi, card)
            want = exact_symbol(seg, 16, card)
            assert want == j - 1
            assert got is None or got == want
