"""GPU parity of exact k-NN query answering against the oracle: neighbour rows bit-exact
(ordered by exact distance, ties by lower row), distances within 1e-5 relative; plus the
approximate-search leaves, the lower-bound candidate sets, ties, host buffers and shapes."""
import numpy as np
import pytest

import planted
from gpu_common import require_gpu, rw, small_dataset, torch
from oracle import index as oindex
from oracle import isax
from oracle import knn as oknn

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.fixture(scope="module")
def built():
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = small_dataset()
    X = torch.from_numpy(x).to(dev)
    idx = P.paris_build(X, 16, 256)
    yield x, X, idx
    idx.free()


def workload_queries(x):
    import synth
    q_rw = synth.random_walk(20, 256, seed=2)                    # independent random walks
    qs, _, _ = synth.sigma_queries(x, x.shape[0], 256, 8)        # 8 per sigma in {0.01, 0.1, 1}
    return np.concatenate([q_rw, qs])


def run_knn(idx, q, k, **kw):
    import paper_2009_00166_gb300 as P
    Q = torch.from_numpy(np.ascontiguousarray(q)).to("cuda")
    i, d = P.paris_exact_knn_ex(idx, Q, k, **kw)[:2]
    torch.cuda.synchronize()
    return i.cpu().numpy(), d.cpu().numpy()


def assert_matches(x, q, k, got_i, got_d):
    want_i, want_d = oknn.knn(x, q, k)
    bad = np.nonzero(~np.all(got_i == want_i, axis=1))[0]
    assert bad.size == 0, f"queries {bad[:5]}: got {got_i[bad[:2]]} want {want_i[bad[:2]]}"
    assert np.allclose(got_d, want_d, rtol=RTOL, atol=0), np.max(np.abs(got_d - want_d) / want_d)


@pytest.mark.parametrize("k", [1, 10])
def test_exact_knn_100k(built, k):
    x, _, idx = built
    q = workload_queries(x)
    gi, gd = run_knn(idx, q, k)
    assert_matches(x, q, k, gi, gd)


def test_exact_knn_chunking_and_stats(built):
    x, _, idx = built
    q = workload_queries(x)[:12]
    a = run_knn(idx, q, 3, chunk=5)
    b = run_knn(idx, q, 3, chunk=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    import paper_2009_00166_gb300 as P
    _, _, st = P.paris_exact_knn_ex(idx, torch.from_numpy(q).cuda(), 3, want_stats=True)
    assert st["candidates"] >= st["refined"] >= 3 * len(q)
    assert st["contenders"] >= 3 * len(q)
    assert st["ms_lbscan"] > 0


def test_host_buffers(built):
    import paper_2009_00166_gb300 as P
    x, _, idx = built
    q = workload_queries(x)[:6]
    oi = np.empty((6, 4), np.int64)
    od = np.empty((6, 4), np.float32)
    P.paris_exact_knn(idx, q, 4, out_idx=oi, out_dist=od)
    assert_matches(x, q, 4, oi, od)


def test_approx_search_leaf_and_seed(built):
    import paper_2009_00166_gb300 as P
    x, X, idx = built
    q = workload_queries(x)
    sax = isax.isax_words(x, 16, 256)
    rows, keys = oindex.sort_order(isax.key64(sax, 256))
    for k in (1, 10):
        leaf, seed = P.paris_approx_search(idx, torch.from_numpy(q).cuda(), k)
        leaf, seed = leaf.cpu().numpy(), seed.cpu().numpy()
        want_d = oknn.knn(x, q, k)[1][:, -1]
        for t in range(q.shape[0]):
            qkey = isax.key128(isax.symbols(isax.paa(q[t], 16)[0], 256), 256) >> 64
            assert tuple(leaf[t]) == oindex.leaf_range(keys, qkey, 2048, k)
            ex, _ = oindex.approx_seed(x, rows, tuple(leaf[t]), q[t], k)
            assert abs(seed[t] - np.ldexp(float(ex), -298)) <= 1e-5 * seed[t]
            assert seed[t] >= want_d[t] ** 2 * (1 - 1e-5)


def test_lb_scan_candidate_set(built):
    import paper_2009_00166_gb300 as P
    x, _, idx = built
    q = workload_queries(x)[[0, 25, 40]]
    sax = isax.isax_words(x, 16, 256)
    for t in range(q.shape[0]):
        pq = isax.paa(q[t], 16)[0]
        lb = isax.mindist_sq(pq, sax, 256, 256)
        thr = float(np.quantile(lb, 0.02))
        rows, lbs, cnt = P.paris_lb_scan(idx, torch.from_numpy(q[t]).cuda(), thr)
        got = set(rows.cpu().numpy().tolist())
        assert cnt == len(got)
        must = set(np.nonzero(lb <= thr * (1 - 1e-4))[0].tolist())
        may = set(np.nonzero(lb <= thr * (1 + 1e-3))[0].tolist())
        assert must <= got <= may
        # the kernel's bound never exceeds the exact MINDIST^2 by more than its stated margin
        r = rows.cpu().numpy()
        assert np.all(lbs.cpu().numpy() <= lb[r] * (1 + 1e-5) + 1e-30)
    # capacity smaller than the candidate count: count reports the total
    rows, _, cnt = P.paris_lb_scan(idx, torch.from_numpy(q[0]).cuda(), 1e9, capacity=100)
    assert cnt == x.shape[0] and rows.numel() == 100


def test_ties_and_duplicates():
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = rw(5000, 256, 9)
    x[4000] = x[17]
    x[4500] = x[17]
    x[10] = x[3000]
    q = np.stack([x[17], x[3000], x[4999]]).astype(np.float32)
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    gi, gd = run_knn(idx, q, 4)
    assert gi[0][:3].tolist() == [17, 4000, 4500]
    assert gi[1][:2].tolist() == [10, 3000]
    assert_matches(x, q, 4, gi, gd)
    idx.free()


def test_fp64_inseparable_near_tie():
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = rw(3000, 256, 10)
    base = x[100].copy()
    a = base.copy()
    a[7] = np.float32(np.nextafter(np.float32(a[7]), np.float32(np.inf)))   # 1 ulp away
    x[2000] = a
    x[2500] = base
    x[100] = x[2999]                       # the query itself is not in the data
    q = base.copy()
    q[50] += np.float32(1e-3)
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    gi, gd = run_knn(idx, q[None], 3)
    assert gi[0][0] == 2500
    assert_matches(x, q[None], 3, gi, gd)
    idx.free()


@pytest.mark.parametrize("length,w,card,leaf", [(128, 16, 256, 2048), (1024, 16, 256, 512),
                                                (256, 8, 16, 64), (96, 16, 256, 16), (256, 16, 256, 1)])
def test_shapes_and_leaf_sizes(length, w, card, leaf):
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    n = 20000 + 37
    x = rw(n, length, 11 + length)
    src = synth.sigma_query_sources(n, 5)
    q = np.concatenate([synth.noisy_queries(x[src], 0.05, [4, 0]), synth.noisy_queries(x[src], 1.0, [4, 2]),
                        rw(3, length, 99)])
    idx = P.paris_build_ex(torch.from_numpy(x).to(dev), w, card, leaf)
    for k in (1, 5):
        gi, gd = run_knn(idx, q, k)
        assert_matches(x, q, k, gi, gd)
    idx.free()


def test_k_equals_n_and_tiny_collections():
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    for n in (1, 2, 7, 33):
        x = rw(n, 256, 40 + n)
        q = rw(3, 256, 80 + n)
        idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
        for k in sorted({1, n}):
            gi, gd = run_knn(idx, q, k)
            assert_matches(x, q, k, gi, gd)
        with pytest.raises(P.ParisError):
            run_knn(idx, q, n + 1)
        idx.free()


def test_bad_queries_rejected(built):
    import paper_2009_00166_gb300 as P
    x, _, idx = built
    q = workload_queries(x)[:2].copy()
    q[1, 3] = np.nan
    with pytest.raises(P.ParisError):
        run_knn(idx, q, 1)
    gi, _ = run_knn(idx, q[:0], 1)
    assert gi.shape == (0, 1)


@pytest.mark.parametrize("length", [1024, 2048])
def test_query_prep_planted_exactness(length):
    """Query PAA (Sec. 3.3.1 query preparation) on queries whose segment 0 has an exact mean just
    below breakpoint 64, 128, 160 or 192: the query word, hence its key and the approximate
    search's leaf, must be the lower region's, and the answers exact."""
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    s = length // 16
    x = rw(8000, length, 60 + length)
    q = rw(12, length, 61 + length)
    beta = isax.breakpoints(256)
    for t in range(12):
        j = (192, 160, 128, 64)[t % 4]
        order = ("plain", "reversed", "shuffled")[t // 4]
        q[t, :s] = planted.below_breakpoint(beta[j - 1], s, order, seed=t)
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    sax = isax.isax_words(x, 16, 256)
    _, keys = oindex.sort_order(isax.key64(sax, 256))
    leaf, _ = P.paris_approx_search(idx, torch.from_numpy(q).to(dev), 1)
    leaf = leaf.cpu().numpy()
    for t in range(q.shape[0]):
        word = isax.symbols(isax.paa(q[t], 16)[0], 256)
        assert word[0] == (192, 160, 128, 64)[t % 4] - 1
        qkey = isax.key128(word, 256) >> 64
        assert tuple(leaf[t]) == oindex.leaf_range(keys, qkey, 2048, 1)
    gi, gd = run_knn(idx, q, 3)
    assert_matches(x, q, 3, gi, gd)
    idx.free()


def test_more_queries_than_a_grid_dimension():
    """70,000 queries in one call (more than the 65,535 blocks of a grid's y extent): every step
    that works per query must cover them all."""
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = rw(3000, 64, 81)
    q = rw(70_000, 64, 82)
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    want_i, want_d = oknn.knn(x, q, 1)
    for mode in (P.PARIS_MODE_BATCHED, P.PARIS_MODE_PLAIN):
        gi, gd = run_knn(idx, q if mode == P.PARIS_MODE_BATCHED else q[-300:], 1, mode=mode)
        wi = want_i if mode == P.PARIS_MODE_BATCHED else want_i[-300:]
        assert np.array_equal(gi, wi)
    leaf, seed = P.paris_approx_search(idx, torch.from_numpy(q).to(dev), 1)
    assert np.all(seed.cpu().numpy() >= want_d[:, 0] ** 2 * (1 - 1e-5))
    idx.free()
