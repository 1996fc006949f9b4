"""Pins of the iSAX oracle (PAA, breakpoints, symbols, key, MINDIST) against values fixed by
the paper's definitions and by mathematics, not by the oracle itself."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import isax

GOLD = os.path.join(os.path.dirname(__file__), "golden", "isax_hand_examples.json")


def phi(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


@pytest.mark.parametrize("card", [2, 4, 8, 16, 64, 256])
def test_breakpoints_quantiles(card):
    b = isax.breakpoints(card)
    assert b.shape == (card - 1,)
    assert np.all(np.diff(b) > 0)
    # symmetric regions, the middle breakpoint at 0
    assert np.array_equal(b, -b[::-1])
    assert b[card // 2 - 1] == 0.0
    # equiprobable under N(0,1): Phi(beta_j) = j / card (erfc is independent of inv_cdf)
    for j, v in enumerate(b, start=1):
        assert abs(phi(v) - j / card) < 2e-15


def test_breakpoints_quartiles_textbook():
    assert np.allclose(isax.breakpoints(4), [-0.6744897501960817, 0.0, 0.6744897501960817], rtol=0, atol=1e-15)
    assert np.allclose(isax.breakpoints(8)[[0, 2]], [-1.1503493803760079, -0.31863936396437514], atol=1e-15)


def test_hand_examples():
    g = json.load(open(GOLD))
    for ex in g["examples"]:
        x = np.array(ex["series"], dtype=np.float32)[None, :]
        p = isax.paa(x, ex["w"])[0]
        assert np.allclose(p, ex["paa"], rtol=0, atol=1e-7)
        s = isax.symbols(p, ex["card"])
        assert s.tolist() == ex["symbols"]
        bits = ex["key_bits"]
        assert isax.key128(s, ex["card"]) == int(bits, 2) << (128 - len(bits))
    for m in g["mindist"]:
        v = isax.mindist_sq(np.array(m["paa_q"]), np.array([m["word"]]), m["n"], m["card"])[0]
        assert abs(v - m["mindist_sq"]) < 1e-14


def test_paa_linear_ramp_closed_form():
    # x_j = a + b*j: the mean of segment i is a + b*(i*s + (s-1)/2)
    n, w = 256, 16
    s = n // w
    a, b = np.float32(-1.25), np.float32(0.0078125)       # exact in fp32, sums exact
    x = (a + b * np.arange(n, dtype=np.float32)).astype(np.float32)
    p = isax.paa(x, w)[0]
    want = [float(a) + float(b) * (i * s + (s - 1) / 2) for i in range(w)]
    assert p.tolist() == want


def test_paa_is_exact_sum_rounded_once():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((50, 64)).astype(np.float32)
    x[3, 5] = np.float32(1e-30)          # tiny values next to large ones
    x[3, 6] = np.float32(-3.0e-38)
    x[7, :8] = np.float32([2.0 ** 60, 1.0, -(2.0 ** 60), 2.0 ** -20, 0, 0, 0, 0])
    p = isax.paa(x, 8)
    for r in range(x.shape[0]):
        for i in range(8):
            exact = sum(Fraction(float(v)) for v in x[r, i * 8:(i + 1) * 8])
            assert p[r, i] == float(exact) / 8       # float(Fraction) rounds correctly once
    # a naive FP64 running sum loses the 1.0 in the planted segment; the oracle does not
    naive = 0.0
    for v in x[7, :8].tolist():
        naive += v
    assert naive == 2.0 ** -20
    assert p[7, 0] == (1.0 + 2.0 ** -20) / 8


def test_paa_planted_segments_exact():
    """Segments whose sum needs every low bit (the planted inputs of the GPU exactness tests):
    the oracle's PAA equals the Fraction sum rounded once / s, and a segment whose exact mean
    sits less than 2^-38/s below breakpoint j takes symbol j - 1."""
    import planted
    beta = isax.breakpoints(256)
    rng = np.random.default_rng(3)
    for s in (32, 64, 128, 256):
        rows = [planted.wide_span(s, rng, v) for v in range(4)]
        rows += [planted.gate(s, span, rng) for span in (10, 12, 15, 16)]
        for j in (64, 128, 160, 192):
            for order in ("plain", "reversed", "shuffled"):
                v = planted.below_breakpoint(beta[j - 1], s, order, seed=j)
                gap = Fraction(float(beta[j - 1])) - planted.exact_mean(v)
                assert 0 < gap <= Fraction(2) ** -38 / s
                p = isax.paa(v[None, :], 1)[0, 0]
                assert isax.symbols(np.array([p]), 256)[0] == j - 1
                rows.append(v)
        for v in rows:
            assert isax.paa(v[None, :], 1)[0, 0] == float(planted.exact_mean(v) * s) / s


def test_symbols_brute_force_and_monotone():
    rng = np.random.default_rng(3)
    card = 256
    b = isax.breakpoints(card)
    v = np.concatenate([rng.standard_normal(2000) * 1.5, b, np.nextafter(b, -np.inf), [-np.inf, np.inf, 0.0, -0.0]])
    s = isax.symbols(v, card)
    for val, sym in zip(v.tolist(), s.tolist()):
        assert sym == sum(1 for t in b.tolist() if t <= val)
    order = np.argsort(v, kind="stable")
    assert np.all(np.diff(s[order].astype(int)) >= 0)


def test_key_root_child_is_first_bits():
    rng = np.random.default_rng(5)
    sym = rng.integers(0, 256, size=(100, 16)).astype(np.uint8)
    k = isax.key64(sym, 256)
    root = (k >> np.uint64(48)).astype(np.int64)
    want = np.zeros(100, np.int64)
    for i in range(16):
        want = want * 2 + (sym[:, i] >> 7)
    assert np.array_equal(root, want)
    # last plane bit of the 64-bit prefix is bit 4 of segment 15
    assert np.array_equal((k & np.uint64(1)).astype(np.int64), ((sym[:, 15] >> 4) & 1).astype(np.int64))


def _rw(nr, n, seed):
    x = np.cumsum(np.random.default_rng(seed).standard_normal((nr, n)), axis=1)
    x = (x - x.mean(1, keepdims=True)) / x.std(1, keepdims=True)
    return x.astype(np.float32)


@pytest.mark.parametrize("card", [4, 256])
def test_mindist_lower_bounds_ed(card):
    n, w = 128, 16
    X = _rw(400, n, 11)
    Q = _rw(20, n, 12)
    sax = isax.isax_words(X, w, card)
    for q in Q:
        pq = isax.paa(q, w)[0]
        lb = isax.mindist_sq(pq, sax, n, card)
        ed = ((X.astype(np.float64) - q.astype(np.float64)) ** 2).sum(1)
        assert np.all(lb <= ed * (1 + 1e-12))
        # never looser than the plain PAA bound (Keogh) pushed through the region edges
        pb = (n / w) * ((isax.paa(X, w) - pq) ** 2).sum(1)
        assert np.all(lb <= pb * (1 + 1e-12))


def test_mindist_zero_against_own_word_and_positive_elsewhere():
    X = _rw(200, 256, 21)
    sax = isax.isax_words(X, 16, 256)
    P = isax.paa(X, 16)
    for r in range(0, 200, 17):
        lb = isax.mindist_sq(P[r], sax, 256, 256)
        assert lb[r] == 0.0
        assert np.sum(lb > 0) >= 150


def test_mindist_approaches_paa_bound_with_cardinality():
    X = _rw(300, 256, 31)
    q = _rw(1, 256, 32)[0]
    pq = isax.paa(q, 16)[0]
    pb = 16 * ((isax.paa(X, 16) - pq) ** 2).sum(1)
    gaps = []
    for card in (4, 16, 256):
        lb = isax.mindist_sq(pq, isax.isax_words(X, 16, card), 256, card)
        gaps.append(float(np.mean(pb - lb)))
    assert gaps[0] > gaps[1] > gaps[2] >= 0
    assert gaps[2] < 0.05 * float(np.mean(pb))
