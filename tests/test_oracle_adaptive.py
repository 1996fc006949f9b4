"""Pins of the adaptive-split leaves of the oracle (Sec. 2.2, ADS+ split rule): a hand-worked
tree, and on random walks the tiling, capacity and shared-prefix invariants plus a brute-force
check that every split is the most balanced one. CPU only."""
import numpy as np
import pytest

from oracle import adaptive, index, isax


def _key64(sym_row, bits):
    """Interleaved key (first 64 bits), written out plane by plane for the test."""
    w = len(sym_row)
    k, nb = 0, 0
    for j in range(bits):
        for i in range(w):
            k = (k << 1) | ((int(sym_row[i]) >> (bits - 1 - j)) & 1)
            nb += 1
    return k << (64 - nb)


def test_hand_worked_split():
    # two segments of 3 bits, leaf capacity 3; all six words share the first bits (1, 0).
    # Second bits: segment 0 -> 0,0,0,1,0,0 (n0=5, n1=1), segment 1 -> 0,1,1,0,1,0 (3, 3):
    # segment 1 splits; the index order is a f b e c d (by interleaved key).
    words = {"a": (4, 0), "b": (4, 2), "c": (5, 2), "d": (6, 0), "e": (4, 3), "f": (5, 0)}
    names = sorted(words, key=lambda n: _key64(words[n], 3))
    assert names == ["a", "f", "b", "e", "c", "d"]
    sym = np.array([words[n] for n in names])
    keys = np.array([_key64(words[n], 3) for n in names], dtype=np.uint64)
    roots, order = adaptive.build(sym, keys, w=2, bits=3, L=3)
    assert list(roots) == [0b10]
    root = roots[0b10]
    assert root.seg == 1
    assert [names[p] for p in order] == ["a", "f", "d", "b", "e", "c"]
    c0, c1 = root.children
    assert (c0.start, c0.count, c0.cards) == (0, 3, (1, 2))
    assert (c1.start, c1.count, c1.cards) == (3, 3, (1, 2))
    # descent: word (6, 0) follows segment 1's second bit 0 to the first leaf
    assert adaptive.descend(roots, (6, 0), _key64((6, 0), 3), 2, 3, 6, 3, 1) == (0, 3)
    # word (7, 7): root 0b11 is empty and no larger root exists -> the last root (0b10); its
    # segment-1 second bit is 1 -> the second leaf
    assert adaptive.descend(roots, (7, 7), _key64((7, 7), 3), 2, 3, 6, 3, 1) == (3, 6)


def _random_tree(n=3000, length=64, L=12, card=256, seed=5):
    import synth
    x = synth.random_walk(n, length, seed=seed)
    sym = isax.isax_words(x, 16, card)
    keys = np.array([isax.key128(s, card) >> 64 for s in sym], dtype=np.uint64)
    rows, ks = index.sort_order(keys)
    roots, order = adaptive.build(sym[rows], ks, w=16, bits=card.bit_length() - 1, L=L)
    return sym[rows], ks, roots, order


def _inner_nodes(roots):
    out = []

    def walk(nd, path_rows):
        out.append(nd)
        if nd.seg >= 0:
            walk(nd.children[0], None)
            walk(nd.children[1], None)

    for r in sorted(roots):
        walk(roots[r], None)
    return out


@pytest.mark.parametrize("L", [5, 12, 40])
def test_random_tree_invariants(L):
    sym, ks, roots, order = _random_tree(L=L)
    N = sym.shape[0]
    assert sorted(order.tolist()) == list(range(N))             # a permutation
    lv = adaptive.leaves(roots)
    pos = 0
    for lf in lv:                                               # leaves tile [0, N) in order
        assert lf.start == pos
        pos += lf.count
        rows = order[lf.start:lf.start + lf.count]
        assert lf.count <= L or all(c == 8 for c in lf.cards)
        for i in range(16):                                     # shared prefix of cards_i bits
            pre = sym[rows, i].astype(np.int64) >> (8 - lf.cards[i])
            assert pre.size == 0 or (pre == pre[0]).all()
    assert pos == N
    # every split is the most balanced among the open segments (lowest index on ties)
    for nd in _inner_nodes(roots):
        if nd.seg < 0:
            continue
        rows = order[nd.start:nd.start + nd.count]
        bal = []
        for i in range(16):
            if nd.cards[i] >= 8:
                bal.append(None)
                continue
            ones = sum((int(sym[r, i]) >> (7 - nd.cards[i])) & 1 for r in rows)
            bal.append(abs(nd.count - 2 * ones))
        best = min(b for b in bal if b is not None)
        assert nd.seg == bal.index(best)
        c0, c1 = nd.children
        assert c0.start == nd.start and c0.count + c1.count == nd.count
        assert nd.count > L


def test_descent_reaches_the_leaf_of_an_equal_word():
    sym, ks, roots, order = _random_tree(L=12)
    N = sym.shape[0]
    lv = adaptive.leaves(roots)
    where = np.empty(N, dtype=np.int64)
    for li, lf in enumerate(lv):
        where[lf.start:lf.start + lf.count] = li
    inv = np.empty(N, dtype=np.int64)
    inv[order] = np.arange(N)
    for p in range(0, N, 97):                                   # query word = a series' word
        lo, hi = adaptive.descend(roots, sym[p], int(ks[p]), 16, 8, N, 12, 1, lv)
        lf = lv[where[inv[p]]]
        assert (lo, hi) == (lf.start, lf.start + min(lf.count, 12))
