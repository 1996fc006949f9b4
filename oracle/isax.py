"""iSAX representation, written out from its definition (test infrastructure only).

Passages followed (ParIS+ paper):
  Sec. 2.2 "iSAX Representation": PAA = mean of each of w equal segments; the y-axis is cut into
    regions, each with a bit-wise symbol; up to 256 symbols (8 bits); a segment takes the symbol
    of the region its PAA value falls in (word 10_2 00_2 11_2 for a 3-segment, 2-bit example).
  Sec. 2.2 "ADS+ Index": the root's children are keyed by the first bit of every segment;
    deeper levels refine one segment by one more bit.
  Sec. 3.3.1: the lower bound between a query PAA and an iSAX word has three branches per
    segment -- PAA above, below or inside the symbol's interval.

Readings where the paper is silent (each also listed in the design notes):
  * regions are equiprobable under N(0,1): breakpoint j of a card-symbol alphabet is
    Phi^-1(j/card), j = 1..card-1, in FP64 (the standard iSAX choice the paper builds on);
  * PAA_i = RN64(exact sum of the s fp32 values of segment i) / s, s = len/w (exactly one
    rounding of the exact sum, then an IEEE division);
  * a PAA equal to a breakpoint belongs to the upper region: symbol = #{j : beta_j <= PAA};
    symbol 0 is the lowest region, so its most significant bit says "PAA >= 0";
  * MINDIST^2 = (n/w) * sum_i d_i^2, d_i = beta_lo - PAA_i (below), PAA_i - beta_hi (above),
    else 0, with beta_lo(0) = -inf and beta_hi(card-1) = +inf;
  * the key interleaves bit planes, most significant plane first: plane j holds bit (b-1-j) of
    segments 0..w-1 in that order, left-aligned in 128 bits; its first w bits are the ADS+ root
    child. Index order uses the top 64 bits.
"""
from __future__ import annotations

import math
from statistics import NormalDist

import numpy as np


def breakpoints(card: int) -> np.ndarray:
    """beta_1..beta_{card-1} = Phi^-1(j/card) in FP64 (Sec. 2.2 regions; equiprobable reading)."""
    assert card >= 2 and card & (card - 1) == 0 and card <= 256
    nd = NormalDist()
    return np.array([nd.inv_cdf(j / card) for j in range(1, card)], dtype=np.float64)


def paa(series: np.ndarray, w: int) -> np.ndarray:
    """PAA of each row: exact segment sum (math.fsum, correctly rounded) divided by s (Sec. 2.2).

    series: [N][n] float32 (or a single row). Returns [N][w] float64.
    """
    x = np.atleast_2d(np.asarray(series, dtype=np.float32))
    n = x.shape[1]
    assert n % w == 0
    s = n // w
    out = np.empty((x.shape[0], w), dtype=np.float64)
    rows = x.astype(np.float64).tolist()
    for r, row in enumerate(rows):
        for i in range(w):
            out[r, i] = math.fsum(row[i * s:(i + 1) * s]) / s
    return out


def symbols(paa_values: np.ndarray, card: int) -> np.ndarray:
    """iSAX symbol per segment: the number of breakpoints <= PAA (upper region on a tie)."""
    beta = breakpoints(card)
    return np.searchsorted(beta, np.asarray(paa_values, dtype=np.float64), side="right").astype(np.uint8)


def isax_words(series: np.ndarray, w: int, card: int) -> np.ndarray:
    """ConvertToSAX (Alg. 2): [N][w] uint8 symbols."""
    return symbols(paa(series, w), card)


def key128(sym_row, card: int) -> int:
    """Bit-plane interleaved key of one word as a Python int (128 bits, left-aligned)."""
    b = card.bit_length() - 1
    w = len(sym_row)
    bits = []
    for j in range(b):                       # plane j = bit (b-1-j) of every segment
        for i in range(w):
            bits.append((int(sym_row[i]) >> (b - 1 - j)) & 1)
    key = 0
    for bit in bits:
        key = (key << 1) | bit
    return key << (128 - len(bits))


def key64(sym: np.ndarray, card: int) -> np.ndarray:
    """Top 64 bits of the interleaved key for every row: [N] uint64."""
    sym = np.atleast_2d(sym)
    return np.array([key128(row, card) >> 64 for row in sym.tolist()], dtype=np.uint64)


def mindist_sq(paa_q: np.ndarray, sym: np.ndarray, n: int, card: int) -> np.ndarray:
    """MINDIST_PAA_iSAX^2 between one query PAA [w] and words [N][w] (Sec. 3.3.1, 3 branches)."""
    beta = breakpoints(card)
    ext = np.concatenate(([-np.inf], beta, [np.inf]))
    sym = np.atleast_2d(sym).astype(np.int64)
    w = sym.shape[1]
    lo = ext[sym]
    hi = ext[sym + 1]
    p = np.asarray(paa_q, dtype=np.float64)[None, :]
    below = p < lo          # PAA BELOW the symbol's interval
    above = p > hi          # PAA ABOVE the interval
    d = np.where(below, lo - p, np.where(above, p - hi, 0.0))
    return (n / w) * (d * d).sum(axis=1)
