"""Index order, approximate search, LB candidate set and exact search (test infrastructure only).

Passages followed (ParIS+ paper):
  Sec. 2.2 ADS+: a tree whose root children are keyed by the first bit of each segment, whose
    nodes refine one segment by one bit, and whose leaves hold at most a capacity of series.
  Sec. 3.3 approximate search: descend to the leaf whose iSAX is most similar to the query's,
    compute the distance to each series there; the minimum is the first BSF.
  Alg. 8 (LBC worker): keep (minDist, position) for every summary with minDist < BSF.
  Alg. 9 (RDC worker): for each kept pair still under BSF, compute the real distance and lower
    BSF when smaller.  Alg. 7 ties these steps together.

  Leaf pruning (ADS+ leaves; applied to in-memory leaves by the MESSI follow-up): every series
    under a tree node has, per segment, a symbol inside the node's range, so the MINDIST from
    the query to the node's box of regions bounds the MINDIST of each of its series.

Readings (also in the design notes):
  * the tree is the fixed-order trie over the bit-plane interleaved key (top 64 bits) stored as
    a sorted array ordered by (key, row); a trie node at depth l is the run of keys sharing
    their first l bits;
  * the approximate leaf: pos = first sorted position whose key >= the query key (clamped to
    the last position), anchor = key at pos; the leaf is the shallowest node containing the
    anchor with at most L' = max(L, k) rows; if it holds fewer than k rows the leaf becomes the k
    consecutive sorted positions starting at its first position (shifted left to fit); if even
    depth 64 holds more than L' rows the leaf is the first L' rows of that node;
  * for k-NN the BSF is the k-th best distance; ties keep the lower row;
  * the pruned units are pages of a fixed number of consecutive rows of the index order (each
    page lies inside the trie node of its common key prefix); a page's box is the per-segment
    range of its rows' symbols.
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


def page_envelopes(sax_in_order: np.ndarray, page_rows: int):
    """Per page of `page_rows` consecutive rows of the index order: the smallest and the largest
    symbol of every segment (the page's box of iSAX regions). Returns (lo, hi), [pages][w]."""
    sym = np.asarray(sax_in_order, dtype=np.int64)
    N, w = sym.shape
    pages = (N + page_rows - 1) // page_rows
    lo = np.empty((pages, w), dtype=np.int64)
    hi = np.empty((pages, w), dtype=np.int64)
    for p in range(pages):
        blk = sym[p * page_rows:(p + 1) * page_rows]
        lo[p] = blk.min(axis=0)
        hi[p] = blk.max(axis=0)
    return lo, hi


def box_mindist_sq(paa_q, lo, hi, n: int, card: int) -> np.ndarray:
    """MINDIST^2 from a query PAA to boxes of iSAX regions (Sec. 2.2 ADS+ nodes and leaves cover
    a region per segment; Sec. 3.3.1's three branches per segment): segment i of a box spans
    symbols lo_i..hi_i, i.e. [beta_lo(lo_i), beta_hi(hi_i)]; d_i is the distance from PAA_i to
    that interval (BELOW / ABOVE / IN), and the bound is (n/w) * sum_i d_i^2."""
    beta = isax.breakpoints(card)
    ext = np.concatenate(([-np.inf], beta, [np.inf]))
    lo = np.atleast_2d(np.asarray(lo, dtype=np.int64))
    hi = np.atleast_2d(np.asarray(hi, dtype=np.int64))
    w = lo.shape[1]
    left = ext[lo]
    right = ext[hi + 1]
    p = np.asarray(paa_q, dtype=np.float64)[None, :]
    d = np.where(p < left, left - p, np.where(p > right, p - right, 0.0))
    return (n / w) * (d * d).sum(axis=1)


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
