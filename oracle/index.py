"""Index order, approximate search, LB candidate set and exact search (test infrastructure only).

Passages followed (ParIS+ paper):
  Sec. 2.2 ADS+: a tree whose root children are keyed by the first bit of each segment, whose
    nodes refine one segment by one bit, and whose leaves hold at most a capacity of series.
  Sec. 3.3 approximate search: descend to the leaf whose iSAX is most similar to the query's,
    compute the distance to each series there; the minimum is the first BSF.
  Alg. 8 (LBC worker): keep (minDist, position) for every summary with minDist < BSF.
  Alg. 9 (RDC worker): for each kept pair still under BSF, compute the real distance and lower
    BSF when smaller.  Alg. 7 ties these steps together.

Readings (also in the design notes):
  * the tree is the fixed-order trie over the bit-plane interleaved key (top 64 bits) stored as
    a sorted array ordered by (key, row); a trie node at depth l is the run of keys sharing
    their first l bits;
  * the approximate leaf: pos = first sorted position whose key >= the query key (clamped to
    the last position), anchor = key at pos; the leaf is the shallowest node containing the
    anchor with at most L' = max(L, k) rows; if it holds fewer than k rows the leaf becomes the k
    consecutive sorted positions starting at its first position (shifted left to fit); if even
    depth 64 holds more than L' rows the leaf is the first L' rows of that node;
  * for k-NN the BSF is the k-th best distance; ties keep the lower row.
"""
from __future__ import annotations

import numpy as np

from . import isax, knn

M64 = (1 << 64) - 1


def sort_order(keys64: np.ndarray):
    """(rows_sorted, keys_sorted): rows ordered by (key, row)."""
    keys64 = np.asarray(keys64, dtype=np.uint64)
    rows = np.lexsort((np.arange(keys64.size), keys64)).astype(np.int64)
    return rows, keys64[rows]


def _hi_mask(l: int) -> int:
    return 0 if l == 0 else (((1 << l) - 1) << (64 - l)) & M64


def node_range(keys_sorted: np.ndarray, anchor: int, l: int):
    """[lo, hi) of sorted positions whose first l key bits equal the anchor's."""
    m = _hi_mask(l)
    lo_key = np.uint64(anchor & m)
    hi_key = np.uint64((anchor | (~m & M64)) & M64)
    lo = int(np.searchsorted(keys_sorted, lo_key, side="left"))
    hi = int(np.searchsorted(keys_sorted, hi_key, side="right"))
    return lo, hi


def leaf_range(keys_sorted: np.ndarray, qkey: int, L: int, k: int):
    """Sorted-position range [lo, hi) of the approximate-search leaf (see module readings)."""
    N = keys_sorted.size
    Lp = max(L, k)
    pos = min(int(np.searchsorted(keys_sorted, np.uint64(qkey), side="left")), N - 1)
    anchor = int(keys_sorted[pos])
    for l in range(65):
        lo, hi = node_range(keys_sorted, anchor, l)
        if hi - lo <= Lp:
            if hi - lo < k:
                s = min(lo, N - k)
                return s, s + k
            return lo, hi
    lo, hi = node_range(keys_sorted, anchor, 64)
    return lo, lo + Lp


def approx_seed(X, rows_sorted, leaf, q, k):
    """Exact k-th best squared distance (scaled int) among the leaf rows, and those rows."""
    lo, hi = leaf
    rows = np.sort(rows_sorted[lo:hi])
    ex = sorted((knn.exact_sq_int(X[r], q), int(r)) for r in rows)
    return ex[k - 1][0], rows


def candidates(paa_q, sax, n, card, bsf_sq: float):
    """Alg. 8 over the whole SAX array: rows whose MINDIST^2 can reach bsf_sq (FP64, ties kept)."""
    lb = isax.mindist_sq(paa_q, sax, n, card)
    return np.nonzero(lb <= bsf_sq * (1.0 + 1e-12))[0], lb


def exact_search(X, sax, keys_sorted, rows_sorted, q, k, L, card):
    """Alg. 7 (approximate search, LBC phase, RDC phase) with exact distances.

    Returns dict(idx, dist, leaf, seed_sq, candidates).
    """
    n = X.shape[1]
    w = sax.shape[1]
    q = np.asarray(q, dtype=np.float32)
    paa_q = isax.paa(q, w)[0]
    qsym = isax.symbols(paa_q, card)
    qkey = isax.key128(qsym, card) >> 64
    leaf = leaf_range(keys_sorted, qkey, L, k)
    seed_int, _ = approx_seed(X, rows_sorted, leaf, q, k)
    seed_sq = float(np.ldexp(float(seed_int), -298))
    cand, lb = candidates(paa_q, sax, n, card, seed_sq)
    # RDC phase: refine candidates in LB order, keeping the k best (exact, row) pairs
    best = []                                   # sorted list of (exact_int, row)
    bsf = seed_int
    for r in cand[np.argsort(lb[cand], kind="stable")]:
        if lb[r] > float(np.ldexp(float(bsf), -298)) * (1.0 + 1e-12):
            continue
        e = knn.exact_sq_int(X[r], q)
        best.append((e, int(r)))
        best.sort()
        best = best[:k]
        if len(best) == k:
            bsf = min(bsf, best[-1][0])
    idx = np.array([r for _, r in best], dtype=np.int64)
    dist = np.sqrt(np.array([np.ldexp(float(e), -298) for e, _ in best]))
    return dict(idx=idx, dist=dist, leaf=leaf, seed_sq=seed_sq, candidates=cand)
