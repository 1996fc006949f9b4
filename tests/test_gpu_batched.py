"""Batched lower-bound scans (a tile of queries per pass over the summaries, FP16 pair tables):
identical exact answers to the plain one-query-per-pass method and to the oracle, for every
query tile, odd batch sizes, both refinement precisions and k in {1, 10}."""
import numpy as np
import pytest

from gpu_common import require_gpu, small_dataset, torch
from oracle import knn as oknn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = small_dataset()
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    q, sig, _ = synth.mixed_sigma_queries(x, x.shape[0], 256, 37)
    q = np.concatenate([q, synth.random_walk(4, 256, seed=2)])
    want = {k: oknn.knn(x, q, k) for k in (1, 10)}
    yield P, idx, q, want
    idx.free()


def x_rows(idx):
    return idx.n


def run(P, idx, q, k, **kw):
    i, d, st = P.paris_exact_knn_ex(idx, torch.from_numpy(q).cuda(), k, want_stats=True, **kw)
    torch.cuda.synchronize()
    return i.cpu().numpy(), d.cpu().numpy(), st


@pytest.mark.parametrize("qt", [0, 2, 4, 8, 12, 16, 24])
@pytest.mark.parametrize("k", [1, 10])
def test_batched_equals_oracle(setup, qt, k):
    P, idx, q, want = setup
    for prec in (P.PARIS_REFINE_FP32, P.PARIS_REFINE_MIXED):
        for prune in (False, True):
            gi, gd, st = run(P, idx, q, k, mode=P.PARIS_MODE_BATCHED, query_tile=qt, precision=prec,
                             leaf_pruning=prune)
            assert st["query_tile"] in (2, 4, 8, 12, 16, 24) and (qt == 0 or st["query_tile"] == qt)
            # at most 16 slots per row group and query pair (a CTA's range end may add a few
            # partial unrolled steps); with leaf pruning, queries that keep few pages take the
            # list scan (no tile lookups) and the tiles visit only kept pages
            full = 16 * (st["query_tile"] // 2) * 32 * ((x_rows(idx) + 31) // 32) * (-(-len(q) // st["query_tile"]))
            assert (0 <= st["lb_lookups"] if prune else 0 < st["lb_lookups"]) and st["lb_lookups"] <= 1.05 * full
            if prune:
                assert st["list_rows"] <= st["pages_kept"] * 256
            else:
                assert st["list_rows"] == 0
            assert np.array_equal(gi, want[k][0])
            assert np.allclose(gd, want[k][1], rtol=1e-5, atol=0)


def test_batched_equals_plain_and_small_chunks(setup):
    P, idx, q, _ = setup
    a = run(P, idx, q, 3, mode=P.PARIS_MODE_PLAIN)
    assert a[2]["lb_lookups"] == 0                       # counted by the batched scans only
    b = run(P, idx, q, 3, mode=P.PARIS_MODE_BATCHED, query_tile=8, chunk=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_bad_query_tile(setup):
    P, idx, q, _ = setup
    with pytest.raises(P.ParisError):
        run(P, idx, q, 1, mode=P.PARIS_MODE_BATCHED, query_tile=6)


def test_pilot_routing_keeps_answers_exact():
    """A collection large enough for the pilot pass (every 128th group of 32 rows): queries whose
    lists would overflow go to the tensor-core screening up front, tight ones are scanned, and
    every answer still equals the oracle's; a tile mixing both kinds is covered by the order."""
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    n = 300_007
    x = synth.random_walk(n, 256, seed=9)
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    src = np.random.default_rng(4).choice(n, 13, replace=False)
    sig = np.array([1.0, 0.01, 1.5, 1.0, 0.1, 2.0, 0.01, 1.0, 1.0, 0.05, 1.2, 1.0, 0.01])
    q = np.stack([synth.noisy_queries(x[src[j:j + 1]], sig[j], [5, j])[0] for j in range(13)])
    for k in (1, 10):
        wi, wd = oknn.knn(x, q, k)
        for qt in (0, 4, 12):
            gi, gd, st = run(P, idx, q, k, mode=P.PARIS_MODE_BATCHED, query_tile=qt, precision=P.PARIS_REFINE_MIXED)
            assert np.array_equal(gi, wi)
            assert np.allclose(gd, wd, rtol=1e-5, atol=0)
            assert st["dense_queries"] >= 1
        fi, fd, _ = run(P, idx, q, k, mode=P.PARIS_MODE_BATCHED, precision=P.PARIS_REFINE_FP32)
        assert np.array_equal(fi, wi) and np.allclose(fd, wd, rtol=1e-5, atol=0)
    idx.free()
