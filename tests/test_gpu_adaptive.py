"""GPU parity of the adaptive-split ADS+ leaves (Sec. 2.2) against the oracle: the tree (every
node's range, split segment and bits per segment) and the leaf order of the series bit-exact,
the approximate-search leaf of every query bit-exact, its seed within 1e-5, and exact answers
with the adaptive seed equal to the oracle's in every query form."""
import numpy as np
import pytest

from gpu_common import require_gpu, rw, torch
from oracle import adaptive as oad
from oracle import index as oindex
from oracle import isax
from oracle import knn as oknn

pytestmark = pytest.mark.gpu


def oracle_tree(x, w, card, L):
    sax = isax.isax_words(x, w, card)
    rows, keys = oindex.sort_order(isax.key64(sax, card))
    bits = card.bit_length() - 1
    roots, order = oad.build(sax[rows], keys, w, bits, L)
    return rows, roots, order


def assert_same_tree(roots, nodes, w):
    seen = set()

    def walk(on, j):
        g = nodes[j]
        seen.add(j)
        assert (g[0], g[1]) == (on.start, on.count), (j, g, on.start, on.count)
        assert tuple(int((g[4] >> (4 * i)) & 15) for i in range(w)) == on.cards
        assert g[2] == on.seg
        if on.seg >= 0:
            walk(on.children[0], int(g[3]))
            walk(on.children[1], int(g[3]) + 1)
        else:
            assert g[3] == -1

    for j, r in enumerate(sorted(roots)):                    # root children first, by word
        walk(roots[r], j)
    assert seen == set(range(nodes.shape[0]))


def query_words(q, w, card):
    sym = isax.isax_words(q, w, card)
    return sym, isax.key64(sym, card)


@pytest.mark.parametrize("length,w,card,L", [(64, 16, 256, 24), (64, 16, 256, 200), (64, 8, 16, 40),
                                             (96, 4, 4, 64)])
def test_tree_and_leaf_order_match_oracle(length, w, card, L):
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = rw(30_011, length, 31)
    X = torch.from_numpy(x).to(dev)
    idx = P.paris_build_ex(X, w, card, leaf_capacity=L)
    P.paris_build_adaptive_leaves(idx)
    info = P.paris_adaptive_leaves_info(idx)
    rows_g, nodes_g = P.paris_adaptive_leaves_export(idx)
    rows, roots, order = oracle_tree(x, w, card, L)
    assert np.array_equal(rows_g.astype(np.int64), rows[order])
    assert_same_tree(roots, nodes_g, w)
    assert info["leaves"] == len(oad.leaves(roots))
    # a second build gives the same tree (the numbering does not depend on scheduling)
    P.paris_build_adaptive_leaves(idx)
    rows2, nodes2 = P.paris_adaptive_leaves_export(idx)
    assert np.array_equal(rows2, rows_g) and np.array_equal(nodes2, nodes_g)
    idx.free()


@pytest.mark.parametrize("k", [1, 7])
def test_descent_leaf_and_seed_match_oracle(k):
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    L, w, card = 48, 16, 256
    x = rw(40_000, 128, 32)
    X = torch.from_numpy(x).to(dev)
    idx = P.paris_build_ex(X, w, card, leaf_capacity=L)
    P.paris_build_adaptive_leaves(idx)
    rows, roots, order = oracle_tree(x, w, card, L)
    lv = oad.leaves(roots)
    qs, _, _ = synth.sigma_queries(x, x.shape[0], 128, 20)    # 20 per sigma in {0.01, 0.1, 1}
    q = np.concatenate([qs, rw(20, 128, 33), -rw(10, 128, 34)])
    leaf, seed = P.paris_approx_search(idx, torch.from_numpy(q).to(dev), k, seed_mode=P.PARIS_SEED_ADAPTIVE)
    leaf, seed = leaf.cpu().numpy(), seed.cpu().numpy()
    sym, keys = query_words(q, w, card)
    want_d = oknn.knn(x, q, k)[1][:, -1]
    leaf_rows = rows[order]
    for t in range(q.shape[0]):
        lo, hi = oad.descend(roots, sym[t], int(keys[t]), w, 8, x.shape[0], L, k, lv)
        assert tuple(leaf[t]) == (lo, hi), t
        ex = sorted(oknn.exact_sq_int(x[r], q[t]) for r in leaf_rows[lo:hi])[k - 1]
        assert abs(seed[t] - np.ldexp(float(ex), -298)) <= 1e-5 * seed[t]
        assert seed[t] >= want_d[t] ** 2 * (1 - 1e-5)
    idx.free()


def test_exact_answers_with_adaptive_seed():
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = rw(50_000, 256, 35)
    X = torch.from_numpy(x).to(dev)
    idx = P.paris_build_ex(X, 16, 256, leaf_capacity=256, bf16_shadow=True)
    P.paris_build_adaptive_leaves(idx)
    qs, _, _ = synth.sigma_queries(x, x.shape[0], 256, 10)
    q = np.concatenate([qs, rw(10, 256, 36)])
    Q = torch.from_numpy(q).to(dev)
    for k in (1, 5):
        want_i, want_d = oknn.knn(x, q, k)
        for mode in (P.PARIS_MODE_PLAIN, P.PARIS_MODE_BATCHED):
            for precision in (P.PARIS_REFINE_FP32, P.PARIS_REFINE_MIXED):
                i, d, st = P.paris_exact_knn_ex(idx, Q, k, mode=mode, precision=precision,
                                                seed=P.PARIS_SEED_ADAPTIVE, want_stats=True)
                assert np.array_equal(i.cpu().numpy(), want_i), (k, mode, precision)
                assert np.allclose(d.cpu().numpy(), want_d, rtol=1e-5, atol=0)
                assert st["leaf_rows"] > 0
    idx.free()


def test_small_and_degenerate_collections():
    """n below the leaf capacity (no split), all-equal words (no segment can split evenly: the
    chain of one-sided splits ends when every bit is fixed), and the seed mode without a tree."""
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = rw(7, 64, 37)
    idx = P.paris_build_ex(torch.from_numpy(x).to(dev), 16, 256, leaf_capacity=16)
    with pytest.raises(P.ParisError):
        P.paris_approx_search(idx, torch.from_numpy(x[:2]).to(dev), 1, seed_mode=P.PARIS_SEED_ADAPTIVE)
    P.paris_build_adaptive_leaves(idx)
    assert P.paris_adaptive_leaves_info(idx)["depth"] == 1
    idx.free()
    # 300 copies of one series plus 40 others, capacity 16: the copies share every bit
    base = rw(41, 64, 38)
    x = np.concatenate([np.repeat(base[:1], 300, axis=0), base[1:]]).astype(np.float32)
    idx = P.paris_build_ex(torch.from_numpy(x).to(dev), 16, 256, leaf_capacity=16)
    P.paris_build_adaptive_leaves(idx)
    rows_g, nodes_g = P.paris_adaptive_leaves_export(idx)
    rows, roots, order = oracle_tree(x, 16, 256, 16)
    assert np.array_equal(rows_g.astype(np.int64), rows[order])
    assert_same_tree(roots, nodes_g, 16)
    big = [lf for lf in oad.leaves(roots) if lf.count >= 300]
    assert len(big) == 1 and all(c == 8 for c in big[0].cards)
    q = x[:3] + np.float32(0.001)
    i, d = P.paris_exact_knn_ex(idx, torch.from_numpy(q).to(dev), 2, seed=P.PARIS_SEED_ADAPTIVE)[:2]
    want_i, want_d = oknn.knn(x, q, 2)
    assert np.array_equal(i.cpu().numpy(), want_i)
    idx.free()
