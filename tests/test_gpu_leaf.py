"""Leaf pruning on the GPU: the page keep-set against the oracle's box MINDIST, no row that the
lower-bound scan keeps is ever in a pruned page, and exact answers with pruning on and off."""
import numpy as np
import pytest

from gpu_common import require_gpu, rw, small_dataset, torch
from oracle import index as oindex
from oracle import isax
from oracle import knn as oknn

pytestmark = pytest.mark.gpu
PAGE = 256


def page_set(bits, npages):
    b = bits.cpu().numpy().view(np.uint32)
    kept = np.nonzero((b[np.arange(npages) // 32] >> (np.arange(npages) % 32).astype(np.uint32)) & 1)[0]
    return set(kept.tolist())


@pytest.mark.parametrize("n", [100_000, 70_001, 200, 1])
def test_leaf_scan_brackets_oracle(n):
    """Kept pages lie between the pages whose exact box MINDIST^2 is <= thr (1 - 1e-4) and those
    <= thr (1 + 1e-3); every row whose exact MINDIST^2 <= thr sits in a kept page."""
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = small_dataset()[:n] if n <= 100_000 else rw(n, 256, 1)
    idx = P.paris_build(torch.from_numpy(np.ascontiguousarray(x)).to(dev), 16, 256)
    _, rows = P.paris_export_order(idx)
    sax = isax.isax_words(x, 16, 256)
    words = sax[rows.astype(np.int64)]
    lo, hi = oindex.page_envelopes(words, PAGE)
    npages = lo.shape[0]
    src = synth.sigma_query_sources(n, 2) if n >= 2 else np.array([0])
    qs = [synth.noisy_queries(x[src], s, [4, j]) for j, s in enumerate((0.01, 0.1, 1.0))]
    q = np.concatenate(qs + [synth.random_walk(2, 256, seed=2)])
    for t in range(q.shape[0]):
        pq = isax.paa(q[t], 16)[0]
        row_lb = isax.mindist_sq(pq, words, 256, 256)
        box = oindex.box_mindist_sq(pq, lo, hi, 256, 256)
        for quant in (0.001, 0.05, 0.5):
            thr = float(np.quantile(row_lb, quant))
            bits, kept = P.paris_leaf_scan(idx, torch.from_numpy(q[t]).to(dev), thr)
            got = page_set(bits, npages)
            assert kept == len(got)
            must = set(np.nonzero(box <= thr * (1 - 1e-4))[0].tolist())
            may = set(np.nonzero(box <= thr * (1 + 1e-3))[0].tolist())
            assert must <= got <= may
            need = set((np.nonzero(row_lb <= thr)[0] // PAGE).tolist())
            assert need <= got
    idx.free()


def run(idx, q, k, **kw):
    import paper_2009_00166_gb300 as P
    i, d, st = P.paris_exact_knn_ex(idx, torch.from_numpy(np.ascontiguousarray(q)).cuda(), k, want_stats=True, **kw)
    torch.cuda.synchronize()
    return i.cpu().numpy(), d.cpu().numpy(), st


@pytest.mark.parametrize("mode", ["plain", "batched"])
@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_knn_with_and_without_pruning(mode, precision):
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = small_dataset()
    idx = P.paris_build_ex(torch.from_numpy(x).to(dev), bf16_shadow=precision == "mixed")
    src = synth.sigma_query_sources(x.shape[0], 6)
    q = np.concatenate([synth.noisy_queries(x[src], s, [4, j]) for j, s in enumerate((0.01, 0.1, 1.0))] +
                       [synth.random_walk(4, 256, seed=2)])
    kw = dict(mode=P.PARIS_MODE_PLAIN if mode == "plain" else P.PARIS_MODE_BATCHED,
              precision=P.PARIS_REFINE_FP32 if precision == "fp32" else P.PARIS_REFINE_MIXED)
    for k in (1, 10):
        wi, wd = oknn.knn(x, q, k)
        on = run(idx, q, k, **kw)
        off = run(idx, q, k, leaf_pruning=False, **kw)
        for gi, gd, st in (on, off):
            assert np.array_equal(gi, wi)
            assert np.allclose(gd, wd, rtol=1e-5, atol=0)
        st_on, st_off = on[2], off[2]
        assert st_off["pages_examined"] == 0 and st_off["pages_kept"] == 0
        assert 0 < st_on["pages_kept"] <= st_on["pages_examined"] == idx_pages(x.shape[0]) * q.shape[0]
        if mode == "plain" and precision == "fp32":
            # a pruned page holds no row the fp32 scan keeps: the candidate sets are the same
            assert st_on["candidates"] == st_off["candidates"]
        else:
            assert st_on["candidates"] <= st_off["candidates"]
    # tight queries keep few pages
    _, _, st = run(idx, q[:6], 1, **kw)
    assert st["pages_kept"] < 0.05 * st["pages_examined"]
    idx.free()


def idx_pages(n):
    return (n + PAGE - 1) // PAGE


@pytest.mark.parametrize("n,length", [(1, 256), (255, 256), (257, 128), (33_333, 1024), (5000, 64)])
def test_pruning_ragged_and_small(n, length):
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = rw(n, length, 90 + n)
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    q = np.concatenate([synth.noisy_queries(x[[0, n // 2, n - 1]], 0.05, [5, 1]), synth.random_walk(2, length, 3)])
    k = min(3, n)
    wi, wd = oknn.knn(x, q, k)
    for mode in (P.PARIS_MODE_PLAIN, P.PARIS_MODE_BATCHED):
        gi, gd, st = run(idx, q, k, mode=mode)
        assert np.array_equal(gi, wi)
        assert np.allclose(gd, wd, rtol=1e-5, atol=0)
        assert st["pages_examined"] == idx_pages(n) * q.shape[0]
    idx.free()
