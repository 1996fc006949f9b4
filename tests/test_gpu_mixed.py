"""Mixed precision (BF16 tensor-core screening + fp32 re-check): identical exact answers to the
FP32 path and to the oracle, on queries whose lower bounds keep many rows (noise sigma >= 1),
with ragged collection sizes, partial query tiles and k up to 16."""
import numpy as np
import pytest

from gpu_common import require_gpu, rw, small_dataset, torch
from oracle import knn as oknn

pytestmark = pytest.mark.gpu


def run(P, idx, q, k, precision, **kw):
    Q = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    i, d, st = P.paris_exact_knn_ex(idx, Q, k, precision=precision, want_stats=True, **kw)
    torch.cuda.synchronize()
    return i.cpu().numpy(), d.cpu().numpy(), st


@pytest.mark.parametrize("k", [1, 10, 16])
def test_mixed_equals_oracle_hard_queries(k):
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = small_dataset()
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    src = synth.sigma_query_sources(x.shape[0], 70)
    q = np.concatenate([synth.noisy_queries(x[src[:60]], 1.5, [9, 0]), synth.noisy_queries(x[src[60:]], 0.05, [9, 1]),
                        synth.random_walk(7, 256, seed=77)])
    gi, gd, st = run(P, idx, q, k, P.PARIS_REFINE_MIXED)
    assert st["dense_queries"] > 0
    fi, fd, _ = run(P, idx, q, k, P.PARIS_REFINE_FP32)
    assert np.array_equal(gi, fi)
    assert np.array_equal(gd, fd)
    want_i, want_d = oknn.knn(x, q, k)
    assert np.array_equal(gi, want_i)
    assert np.allclose(gd, want_d, rtol=1e-5, atol=0)
    idx.free()


@pytest.mark.parametrize("n,length", [(30001, 256), (20000 + 63, 128), (9000, 64), (12001, 512), (20011, 320),
                                      (16411, 1024)])
def test_mixed_ragged_shapes(n, length):
    """Longer series put fewer queries in a screening group (256 up to len 256, then
    65536 / len rounded down to a multiple of 32: 192 at 320, 128 at 512, 64 at 1024), so 131
    queries span one to three groups; k = 3 at len > 256 runs without the threshold pass."""
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = rw(n, length, 300 + length)
    src = synth.sigma_query_sources(n, 131)
    q = synth.noisy_queries(x[src], 2.0, [10, length])          # 131 queries: one full and one partial tile
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    for k in (1, 3):
        gi, gd, st = run(P, idx, q, k, P.PARIS_REFINE_MIXED, chunk=200)
        assert st["dense_queries"] > 0
        want_i, want_d = oknn.knn(x, q, k)
        assert np.array_equal(gi, want_i)
        assert np.allclose(gd, want_d, rtol=1e-5, atol=0)
    idx.free()


def test_mixed_falls_back_when_unsupported():
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x = rw(5000, 96, 5)                                          # len not a multiple of 64
    q = rw(4, 96, 6)
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    gi, gd, st = run(P, idx, q, 2, P.PARIS_REFINE_MIXED)
    assert st["dense_queries"] == 0
    assert np.array_equal(gi, oknn.knn(x, q, 2)[0])
    idx.free()


@pytest.mark.parametrize("length", [64, 128, 256])
def test_shadow_written_by_encode_pass(length):
    """bf16_shadow=1 builds the screening's inputs in the encode pass: same exact answers as an
    index whose inputs are built by its first mixed-precision query."""
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    n = 150_001
    x = rw(n, length, 17)
    q, _, _ = synth.mixed_sigma_queries(x, n, length, 30, 0.5, 2.0, seed=8)
    X = torch.from_numpy(x).to(dev)
    fused = P.paris_build_ex(X, bf16_shadow=True)
    lazy = P.paris_build_ex(X)
    wi, wd = oknn.knn(x, q, 5)
    for idx in (fused, lazy):
        gi, gd, st = run(P, idx, q, 5, P.PARIS_REFINE_MIXED, mode=P.PARIS_MODE_BATCHED)
        assert np.array_equal(gi, wi)
        assert np.allclose(gd, wd, rtol=1e-5, atol=0)
        assert st["dense_queries"] > 0
    fused.free()
    lazy.free()
