"""Adaptive-split ADS+ leaves (test infrastructure only: never imported by the library).

Passage followed (ParIS+ paper, Sec. 2.2, ADS+ index): the root has one child per combination of
the first bit of every segment; a leaf that holds more series than the leaf capacity becomes an
inner node with two children, obtained by raising the cardinality of one segment by one bit,
namely the segment whose extra bit divides the node's series into the two most balanced parts.
The approximate search (Sec. 3.3) follows the query's iSAX bits down to a leaf and seeds the
best-so-far with the distances to that leaf's series.

Readings (also in the design notes):
  * the series start in the index order (sorted by (interleaved key, row)); a split keeps the
    order of each side (stable), bit 0 before bit 1, so the leaves tile the series in
    depth-first order and root children come in increasing order of their first-bit word;
  * "most balanced" is the smallest |n0 - n1| over the segments that still have a bit to add;
    ties go to the lowest segment index; a split that leaves one side empty is still made
    (the empty side is an empty leaf); a node whose segments all have every bit stays a leaf
    of any size;
  * descent: a root child that holds no series is replaced by the first non-empty root child
    with a larger first-bit word, else the last non-empty one; an empty leaf is replaced by
    the leaf that holds the series at the empty leaf's start position (the last series when it
    starts past the end); like the fixed-order trie, a leaf with fewer than k series becomes
    the k consecutive series starting at its first one (shifted left to fit), and a leaf with
    more than L' = max(L, k) series is cut to its first L'.
  * parity unpinned by a printed example: the paper gives the split rule in words only; the
    tests pin the construction by its invariants (tiling, capacity, shared prefixes, and a
    brute-force check that every split is the most balanced one).
"""
from __future__ import annotations

import numpy as np


class Node:
    __slots__ = ("start", "count", "cards", "seg", "children", "root")

    def __init__(self, start, count, cards, root=-1):
        self.start = start          # first position of the node's series in the leaf order
        self.count = count          # number of series under the node
        self.cards = cards          # bits of each segment's symbol fixed by the path (tuple)
        self.seg = -1               # split segment (-1: leaf)
        self.children = None        # (bit-0 child, bit-1 child)
        self.root = root            # first-bit word of a root child (-1 below the root)


def _bit(sym, seg, card_bits, total_bits):
    """The next bit of segment `seg` below the `card_bits` already fixed."""
    return (sym[:, seg].astype(np.int64) >> (total_bits - 1 - card_bits)) & 1


def build(sym_in_order: np.ndarray, keys_in_order: np.ndarray, w: int, bits: int, L: int):
    """Adaptive-split tree over the series in index order.

    sym_in_order: [N][w] symbols of the series in index order; keys_in_order: their 64-bit
    interleaved keys (the first w bits are the first bit of every segment). Returns
    (roots, order): roots maps each non-empty first-bit word to its root child, and order[j] is
    the index-order position of the j-th series in leaf order.
    """
    sym = np.asarray(sym_in_order, dtype=np.int64)
    keys = np.asarray(keys_in_order, dtype=np.uint64)
    N = sym.shape[0]
    rootw = (keys >> np.uint64(64 - w)).astype(np.int64)
    order = []
    roots = {}

    def grow(node, pos):
        # pos: index-order positions of the node's series, in the node's order
        if len(pos) <= L:
            order.extend(pos.tolist())
            return
        open_segs = [i for i in range(w) if node.cards[i] < bits]
        if not open_segs:
            order.extend(pos.tolist())
            return
        best, best_bal = -1, None
        for i in open_segs:
            ones = int(_bit(sym[pos], i, node.cards[i], bits).sum())
            bal = abs(len(pos) - 2 * ones)
            if best_bal is None or bal < best_bal:
                best, best_bal = i, bal
        b = _bit(sym[pos], best, node.cards[best], bits)
        p0, p1 = pos[b == 0], pos[b == 1]
        cards = list(node.cards)
        cards[best] += 1
        c0 = Node(node.start, len(p0), tuple(cards))
        c1 = Node(node.start + len(p0), len(p1), tuple(cards))
        node.seg = best
        node.children = (c0, c1)
        grow(c0, p0)
        grow(c1, p1)

    start = 0
    for r in np.unique(rootw):
        pos = np.nonzero(rootw == r)[0]
        node = Node(start, len(pos), tuple([1] * w), root=int(r))
        roots[int(r)] = node
        grow(node, pos)
        start += len(pos)
    assert len(order) == N
    return roots, np.asarray(order, dtype=np.int64)


def leaves(roots):
    """All leaves in depth-first order."""
    out = []

    def walk(nd):
        if nd.seg < 0:
            out.append(nd)
        else:
            walk(nd.children[0])
            walk(nd.children[1])

    for r in sorted(roots):
        walk(roots[r])
    return out


def descend(roots, qsym, qkey: int, w: int, bits: int, N: int, L: int, k: int, leaf_list=None):
    """Leaf-order range [lo, hi) of the query's approximate-search leaf (module readings)."""
    r = int(qkey) >> (64 - w)
    ids = sorted(roots)
    bigger = [x for x in ids if x >= r]
    node = roots[bigger[0] if bigger else ids[-1]]
    while node.seg >= 0:
        i = node.seg
        b = (int(qsym[i]) >> (bits - 1 - node.cards[i])) & 1
        node = node.children[b]
    lo, cnt = node.start, node.count
    if cnt == 0:
        p = min(lo, N - 1)
        for lf in (leaf_list if leaf_list is not None else leaves(roots)):
            if lf.count > 0 and lf.start <= p < lf.start + lf.count:
                lo, cnt = lf.start, lf.count
                break
    Lp = max(L, k)
    if cnt < k:
        lo = min(lo, N - k)
        return lo, lo + k
    if cnt > Lp:
        return lo, lo + Lp
    return lo, lo + cnt
