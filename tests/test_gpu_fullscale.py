"""Parity at the full workload: 20M x 256 random-walk series, 1000 noisy queries per noise
level sigma in {0.01, 0.1, 1.0}, answered in one call by the batched scan with mixed-precision
refinement (the launch configuration the benchmark times). Sampled queries are compared with
the oracle's exact search over the whole collection; for every query, the reported distance is
checked against the exact distance of the reported row, and it may not exceed the distance of
the source row the query was made from (an upper bound on the nearest neighbour's)."""
import numpy as np
import pytest

from gpu_common import require_gpu, torch
from oracle import knn as oknn

pytestmark = pytest.mark.gpu

N, LEN, PER_SIGMA = 20_000_000, 256, 1000


@pytest.fixture(scope="module")
def full():
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    free, _ = torch.cuda.mem_get_info()
    if free < 48e9:
        pytest.skip("needs about 48 GB of free device memory")
    x = np.empty((N, LEN), np.float32)
    synth.random_walk(N, LEN, seed=1, out=x)
    q, sig, src = synth.sigma_queries(x, N, LEN, PER_SIGMA)
    X = torch.from_numpy(x).to(dev)
    idx = P.paris_build(X, 16, 256)
    yield P, idx, x, q, sig, src
    idx.free()
    del X
    torch.cuda.empty_cache()


def test_full_workload_every_query_consistent(full):
    P, idx, x, q, sig, src = full
    Q = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    gi, gd, st = P.paris_exact_knn_ex(idx, Q, 1, mode=P.PARIS_MODE_BATCHED, precision=P.PARIS_REFINE_MIXED,
                                      want_stats=True)
    gi, gd = gi.cpu().numpy()[:, 0], gd.cpu().numpy()[:, 0]
    assert np.all((gi >= 0) & (gi < N))
    # exact distance of the reported row, FP64 from the fp32 inputs
    exact = np.sqrt(((x[gi].astype(np.float64) - q.astype(np.float64)) ** 2).sum(axis=1))
    assert np.allclose(gd, exact, rtol=1e-5, atol=1e-6)
    # the source row is a candidate: the nearest neighbour is no farther
    via_src = np.sqrt(((x[src].astype(np.float64) - q.astype(np.float64)) ** 2).sum(axis=1))
    assert np.all(exact <= via_src * (1 + 1e-12))
    assert st["dense_queries"] > 0          # the loose queries went through the tensor-core path


@pytest.mark.parametrize("k", [1, 10])
def test_full_workload_sampled_against_oracle(full, k):
    P, idx, x, q, sig, src = full
    pick = np.array([3, 777, 1000 + 5, 1000 + 901, 2000 + 17, 2000 + 640])  # two per noise level
    Q = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    gi, gd = P.paris_exact_knn_ex(idx, Q, k, mode=P.PARIS_MODE_BATCHED, precision=P.PARIS_REFINE_MIXED)
    gi, gd = gi.cpu().numpy()[pick], gd.cpu().numpy()[pick]
    wi, wd = oknn.knn_chunked(lambda a, b: x[a:b], N, q[pick], k)
    assert np.array_equal(gi, wi)
    assert np.allclose(gd, wd, rtol=1e-5, atol=0)
