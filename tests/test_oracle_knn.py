"""Pins of the exact k-NN oracle and of the index/approximate-search oracle: brute force with
exact rational arithmetic on tiny inputs, planted ties and near ties, and the paper's claim that
exact search (Alg. 7) returns the brute-force answer."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import index, isax, knn


def frac_sq(x, q):
    return sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(x, q))


def brute(X, q, k):
    d = sorted((frac_sq(X[r], q), r) for r in range(X.shape[0]))
    return [r for _, r in d[:k]], [float(v) ** 0.5 for v, _ in d[:k]]


def _rw(nr, n, seed):
    x = np.cumsum(np.random.default_rng(seed).standard_normal((nr, n)), axis=1)
    x = (x - x.mean(1, keepdims=True)) / x.std(1, keepdims=True)
    return x.astype(np.float32)


def test_exact_sq_int_matches_fractions():
    X = _rw(5, 64, 1)
    X[0, 3] = np.float32(1e-40)            # subnormal
    X[1, 0] = np.float32(3e38)
    q = _rw(1, 64, 2)[0]
    for r in range(5):
        assert Fraction(knn.exact_sq_int(X[r], q), 2 ** 298) == frac_sq(X[r], q)


@pytest.mark.parametrize("k", [1, 3, 7])
def test_knn_equals_brute_force(k):
    X = _rw(60, 32, 3)
    X[17] = X[5]                           # exact duplicates: equal distance, lower row first
    X[40] = X[5]
    Q = np.concatenate([_rw(4, 32, 4), X[5:6]])
    idx, dist = knn.knn(X, Q, k)
    for t in range(Q.shape[0]):
        bi, bd = brute(X, Q[t], k)
        assert idx[t].tolist() == bi
        assert np.allclose(dist[t], bd, rtol=1e-15)
    assert idx[-1][:min(k, 3)].tolist() == [5, 17, 40][:min(k, 3)]


def test_knn_resolves_fp64_near_tie_exactly():
    n = 16
    X = np.zeros((4, n), np.float32)
    X[:, 0] = 1.0
    X[1, 1] = np.float32(2.0 ** -30)        # E = 1 + 2^-60: rounds to 1.0 in FP64
    X[2, 0] = np.float32(1.0 + 2.0 ** -23)  # clearly farther
    X[3, 0] = 2.0
    q = np.zeros(n, np.float32)
    # rows 0 and 1 at FP64 1.0 (row 1 exactly farther), row 0 wins; move row 0 after row 1:
    X = X[[1, 0, 2, 3]]
    d64 = ((X.astype(np.float64) - q) ** 2).sum(1)
    assert d64[0] == d64[1]                 # FP64 cannot separate them
    idx, _ = knn.knn(X, q[None], 2)
    assert idx[0].tolist() == [1, 0]        # exact order: 1.0 < 1 + 2^-60
    assert brute(X, q, 2)[0] == [1, 0]


def test_knn_chunked_equals_knn():
    X = _rw(3000, 64, 5)
    Q = np.concatenate([_rw(3, 64, 6), X[[10, 2500]] + np.float32(0.01)])
    a = knn.knn(X, Q, 5)
    b = knn.knn_chunked(lambda r0, r1: X[r0:r1], X.shape[0], Q, 5, chunk=700)
    assert np.array_equal(a[0], b[0])
    assert np.allclose(a[1], b[1], rtol=1e-15)


def _brute_leaf(keys_sorted, qkey, L, k):
    N = keys_sorted.size
    ks = [int(v) for v in keys_sorted]
    pos = next((i for i, v in enumerate(ks) if v >= qkey), N - 1)
    a = ks[pos]
    Lp = max(L, k)
    for l in range(65):
        members = [i for i, v in enumerate(ks) if (v >> (64 - l) if l else 0) == (a >> (64 - l) if l else 0)]
        if len(members) <= Lp:
            lo, hi = members[0], members[-1] + 1
            assert hi - lo == len(members)          # a trie node is a contiguous run
            if hi - lo < k:
                s = min(lo, N - k)
                return s, s + k
            return lo, hi
    members = [i for i, v in enumerate(ks) if v == a]
    return members[0], members[0] + Lp


def test_leaf_range_brute_force():
    rng = np.random.default_rng(9)
    X = _rw(500, 64, 7)
    sax = isax.isax_words(X, 16, 256)
    rows, keys = index.sort_order(isax.key64(sax, 256))
    # sorted by (key, row)
    assert all((int(keys[i]), rows[i]) < (int(keys[i + 1]), rows[i + 1]) for i in range(499))
    dup = np.concatenate([keys[:5], np.repeat(keys[5], 40), keys[6:]])   # a run of equal keys
    for L, k in [(8, 1), (32, 10), (3, 5), (1, 1), (16, 20)]:
        for _ in range(25):
            qk = int(rng.integers(0, 2 ** 63, dtype=np.int64)) * 2 + int(rng.integers(0, 2))
            assert index.leaf_range(keys, qk, L, k) == _brute_leaf(keys, qk, L, k)
        for qk in (0, int(keys[0]), int(keys[250]), int(keys[-1]), 2 ** 64 - 1):
            assert index.leaf_range(keys, qk, L, k) == _brute_leaf(keys, qk, L, k)
        assert index.leaf_range(dup, int(keys[5]), L, k) == _brute_leaf(dup, int(keys[5]), L, k)


@pytest.mark.parametrize("k", [1, 10])
def test_exact_search_reaches_brute_force(k):
    X = _rw(4000, 128, 8)
    sax = isax.isax_words(X, 16, 256)
    rows, keys = index.sort_order(isax.key64(sax, 256))
    base = X[[3, 1200, 3999]]
    Q = np.concatenate([_rw(2, 128, 10), (base + 0.05 * np.random.default_rng(1).standard_normal(base.shape)).astype(np.float32)])
    want = knn.knn(X, Q, k)
    for t in range(Q.shape[0]):
        res = index.exact_search(X, sax, keys, rows, Q[t], k, L=64, card=256)
        assert res["idx"].tolist() == want[0][t].tolist()
        assert np.allclose(res["dist"], want[1][t], rtol=1e-15)
        # the approximate-search seed is an upper bound of the exact k-th distance
        assert res["seed_sq"] >= want[1][t][-1] ** 2 * (1 - 1e-12)
        # pruning never removes an answer row
        assert set(want[0][t].tolist()) <= set(res["candidates"].tolist())


def test_box_mindist_hand_value_and_special_cases():
    """MINDIST to a box of iSAX regions: a hand-computed 2-segment, 4-symbol case; a box of one
    word equals that word's MINDIST; a box spanning every symbol gives 0."""
    from statistics import NormalDist
    b1 = NormalDist().inv_cdf(0.25)                      # breakpoints -0.674.., 0, 0.674..
    # segment 0 spans symbols 0..1 (PAA <= 0): PAA 1.0 lies 1.0 above it;
    # segment 1 spans symbols 1..3 (PAA >= b1): PAA -1.0 lies b1 + 1.0 below it
    got = index.box_mindist_sq(np.array([1.0, -1.0]), [[0, 1]], [[1, 3]], 8, 4)[0]
    want = (8 / 2) * (1.0 ** 2 + (b1 - (-1.0)) ** 2)
    assert abs(got - want) <= 1e-15 * want
    rng = np.random.default_rng(4)
    words = rng.integers(0, 256, (50, 16))
    paa_q = rng.standard_normal(16)
    assert np.array_equal(index.box_mindist_sq(paa_q, words, words, 256, 256),
                          isax.mindist_sq(paa_q, words, 256, 256))
    assert index.box_mindist_sq(paa_q, np.zeros((1, 16), int), np.full((1, 16), 255), 256, 256)[0] == 0.0


def test_page_envelopes_bound_every_row():
    """Envelopes hold every row's symbols and attain their ends; a page's box MINDIST is a lower
    bound of each of its rows' MINDIST (hence of their distances), reached by a one-row page;
    widening a box never raises its bound."""
    x = _rw(3000, 64, 31)
    sax = isax.isax_words(x, 16, 256)
    rows, _ = index.sort_order(isax.key64(sax, 256))
    words = sax[rows]
    for P in (1, 32, 256, 1000):
        lo, hi = index.page_envelopes(words, P)
        assert lo.shape[0] == -(-3000 // P)
        for p in range(lo.shape[0]):
            blk = words[p * P:(p + 1) * P].astype(int)
            assert np.all(blk >= lo[p]) and np.all(blk <= hi[p])
            for i in range(16):
                assert lo[p, i] in blk[:, i] and hi[p, i] in blk[:, i]
    q = _rw(5, 64, 32)
    lo, hi = index.page_envelopes(words, 64)
    for t in range(q.shape[0]):
        pq = isax.paa(q[t], 16)[0]
        box = index.box_mindist_sq(pq, lo, hi, 64, 256)
        row_lb = isax.mindist_sq(pq, words, 64, 256)
        ed2 = ((x[rows].astype(np.float64) - q[t]) ** 2).sum(axis=1)
        for p in range(lo.shape[0]):
            seg = slice(p * 64, (p + 1) * 64)
            assert box[p] <= row_lb[seg].min() + 1e-12
            assert box[p] <= ed2[seg].min() + 1e-9
        wide = index.box_mindist_sq(pq, np.maximum(lo - 3, 0), np.minimum(hi + 3, 255), 64, 256)
        assert np.all(wide <= box)
    one_lo, one_hi = index.page_envelopes(words, 1)
    assert np.array_equal(index.box_mindist_sq(isax.paa(q[0], 16)[0], one_lo, one_hi, 64, 256),
                          isax.mindist_sq(isax.paa(q[0], 16)[0], words, 64, 256))
