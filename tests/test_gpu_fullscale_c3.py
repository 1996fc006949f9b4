"""Parity at full size for the batch workload: 50M x 256 random-walk series, one batch of 4096
queries with noise sigma ~ U[0.01, 2], k in {1, 10}, batched scan with mixed-precision
refinement. Sampled queries are compared with the oracle's exact search over the whole
collection; every query's reported distances are checked against the exact distances of the
reported rows (ascending, and no farther than the source row the query was made from)."""
import numpy as np
import pytest

from gpu_common import require_gpu, torch
from oracle import knn as oknn

pytestmark = pytest.mark.gpu

N, LEN, BATCH = 50_000_000, 256, 4096


@pytest.fixture(scope="module")
def full():
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    free, _ = torch.cuda.mem_get_info()
    if free < 100e9:
        pytest.skip("needs about 100 GB of free device memory")
    x = np.empty((N, LEN), np.float32)
    synth.random_walk(N, LEN, seed=1, out=x)
    q, sig, src = synth.mixed_sigma_queries(x, N, LEN, BATCH, 0.01, 2.0, seed=5)
    X = torch.from_numpy(x).to(dev)
    idx = P.paris_build(X, 16, 256)
    yield P, idx, x, np.ascontiguousarray(q), src
    idx.free()
    del X
    torch.cuda.empty_cache()


@pytest.mark.parametrize("k", [1, 10])
def test_batch_of_4096(full, k):
    P, idx, x, q, src = full
    Q = torch.from_numpy(q).cuda()
    gi, gd = P.paris_exact_knn_ex(idx, Q, k, mode=P.PARIS_MODE_BATCHED, precision=P.PARIS_REFINE_MIXED)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    assert np.all(np.diff(gd, axis=1) >= 0)
    rows = gi.reshape(-1)
    qq = np.repeat(q, k, axis=0).astype(np.float64)
    exact = np.sqrt(((x[rows].astype(np.float64) - qq) ** 2).sum(axis=1)).reshape(gi.shape)
    assert np.allclose(gd, exact, rtol=1e-5, atol=1e-6)
    via_src = np.sqrt(((x[src].astype(np.float64) - q.astype(np.float64)) ** 2).sum(axis=1))
    assert np.all(exact[:, 0] <= via_src * (1 + 1e-12))
    pick = np.array([0, 1111, 2500, 4095])
    wi, wd = oknn.knn_chunked(lambda a, b: x[a:b], N, q[pick], k)
    assert np.array_equal(gi[pick], wi)
    assert np.allclose(gd[pick], wd, rtol=1e-5, atol=0)
