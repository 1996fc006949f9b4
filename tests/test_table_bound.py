"""CPU check of the lower-bound table's rounding (no GPU): each entry is formed in fp32 from the
FP64 PAA and region ends held between their fp32 roundings down and up, the distance rounded
toward -inf, then squared and scaled with rounding toward -inf. The emulation below (numpy fp32,
each result moved one step down, at least as low as directed rounding) must never exceed the
exact (len/w) * distance^2 of the FP64 values, for random PAA values, values on and next to
every region end, and every symbol."""
from fractions import Fraction

import numpy as np

from oracle import isax

F32 = np.float32


def down(x):
    return np.nextafter(F32(x), F32(-np.inf))


def table_entry(P, lo, hi, scale):
    p_lo = F32(P) if float(F32(P)) <= P else down(F32(P))
    p_hi = F32(P) if float(F32(P)) >= P else np.nextafter(F32(P), F32(np.inf))
    lo_d = F32(lo) if np.isinf(lo) or float(F32(lo)) <= lo else down(F32(lo))
    hi_u = F32(hi) if np.isinf(hi) or float(F32(hi)) >= hi else np.nextafter(F32(hi), F32(np.inf))
    d = F32(0.0)
    if p_hi < lo_d:
        d = down(lo_d - p_hi)
    elif p_lo > hi_u:
        d = down(p_lo - hi_u)
    return down(down(d * d) * F32(scale))


def exact_entry(P, lo, hi, scale):
    if P < lo:
        d = Fraction(lo) - Fraction(P)
    elif P > hi:
        d = Fraction(P) - Fraction(hi)
    else:
        return Fraction(0)
    return scale * d * d


def test_entries_never_exceed_the_exact_bound():
    card, scale = 256, 16
    beta = isax.breakpoints(card)
    ext = np.concatenate(([-np.inf], beta, [np.inf]))
    rng = np.random.default_rng(7)
    paa = list(rng.normal(0, 1.2, 300))
    for b in beta[::17]:                       # on and next to region ends
        paa += [b, np.nextafter(b, np.inf), np.nextafter(b, -np.inf), b + 1e-9, b - 1e-9]
    tight = 0
    for P in paa:
        for c in range(card):
            lo, hi = ext[c], ext[c + 1]
            t = table_entry(P, lo, hi, scale)
            ex = exact_entry(P, lo, hi, scale)
            assert Fraction(float(t)) <= ex
            if ex > 0 and Fraction(float(t)) >= ex * (1 - Fraction(1, 1 << 20)):
                tight += 1
    assert tight > 0.9 * sum(1 for P in paa for c in range(card) if exact_entry(P, ext[c], ext[c + 1], scale) > 0)
