"""Several collections in one call (paris_exact_knn_multi): series lengths 128, 256 and 1024,
one batched lower-bound scan launch per chunk round shared by all collections. Every answer
equals the oracle's on its own collection and the single-collection call's, for both refinement
precisions, k in {1, 10}, every query tile, a collection without queries, small chunks (several
rounds, collections running out of chunks at different rounds) and a collection large enough
for the pilot pass."""
import numpy as np
import pytest

from gpu_common import require_gpu, rw, torch
from oracle import knn as oknn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def colls():
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    shapes = [(40_003, 128, 11), (20_011, 256, 12), (5_003, 1024, 13)]
    xs, idxs, qs = [], [], []
    for j, (n, length, seed) in enumerate(shapes):
        x = rw(n, length, seed)
        xs.append(x)
        idxs.append(P.paris_build(torch.from_numpy(x).to(dev), 16, 256))
        q, _, _ = synth.mixed_sigma_queries(x, n, length, 9 + 4 * j, 0.01, 2.0, seed=20 + j)
        qs.append(np.ascontiguousarray(q))
    want = {k: [oknn.knn(x, q, k) for x, q in zip(xs, qs)] for k in (1, 10)}
    yield P, idxs, xs, qs, want
    for ix in idxs:
        ix.free()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("k", [1, 10])
@pytest.mark.parametrize("qt", [0, 4, 12])
def test_multi_equals_oracle(colls, precision, k, qt):
    P, idxs, xs, qs, want = colls
    prec = P.PARIS_REFINE_FP32 if precision == "fp32" else P.PARIS_REFINE_MIXED
    Q = [torch.from_numpy(q).cuda() for q in qs]
    outs, stats = P.paris_exact_knn_multi(idxs, Q, k, query_tile=qt, precision=prec, want_stats=True)
    for c, (gi, gd) in enumerate(outs):
        wi, wd = want[k][c]
        assert np.array_equal(gi.cpu().numpy(), wi), c
        assert np.allclose(gd.cpu().numpy(), wd, rtol=1e-5, atol=0), c
        assert stats[c]["query_tile"] in (2, 4, 8, 12, 16, 24)
        single = P.paris_exact_knn_ex(idxs[c], Q[c], k, mode=P.PARIS_MODE_BATCHED, precision=prec)
        assert np.array_equal(single[0].cpu().numpy(), wi)


def test_multi_rounds_and_empty_collection(colls):
    P, idxs, xs, qs, want = colls
    Q = [torch.from_numpy(q).cuda() for q in qs]
    Q[1] = Q[1][:0]                                        # no queries for the middle collection
    outs = P.paris_exact_knn_multi(idxs, Q, 10, chunk=3)  # 3 queries per chunk: several rounds
    for c in (0, 2):
        assert np.array_equal(outs[c][0].cpu().numpy(), want[10][c][0])
    assert outs[1][0].shape == (0, 10)
    plain = P.paris_exact_knn_multi(idxs[:1], Q[:1], 1, mode=P.PARIS_MODE_PLAIN)
    assert np.array_equal(plain[0][0].cpu().numpy(), want[1][0][0])


def test_multi_rejects_bad_arguments(colls):
    P, idxs, xs, qs, _ = colls
    Q = [torch.from_numpy(q).cuda() for q in qs]
    with pytest.raises(P.ParisError):
        P.paris_exact_knn_multi(idxs + idxs[:2], Q + Q[:2], 1)      # more than 4 collections
    x = rw(3000, 128, 5)
    other = P.paris_build(torch.from_numpy(x).cuda(), 16, 64)     # another cardinality
    with pytest.raises(P.ParisError):
        P.paris_exact_knn_multi([idxs[0], other], [Q[0], Q[0]], 1)
    other.free()


def test_multi_with_pilot_pass():
    """One collection above the pilot pass's size, sharing the launch with a small one."""
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    big = rw(300_007, 128, 31)
    small = rw(9_001, 256, 32)
    ib = P.paris_build(torch.from_numpy(big).to(dev), 16, 256)
    isml = P.paris_build(torch.from_numpy(small).to(dev), 16, 256)
    qb, _, _ = synth.mixed_sigma_queries(big, big.shape[0], 128, 14, 0.01, 2.0, seed=40)
    qsm, _, _ = synth.mixed_sigma_queries(small, small.shape[0], 256, 5, 0.01, 2.0, seed=41)
    outs, stats = P.paris_exact_knn_multi([ib, isml], [torch.from_numpy(qb).cuda(), torch.from_numpy(qsm).cuda()],
                                          1, precision=P.PARIS_REFINE_MIXED, want_stats=True)
    for (gi, gd), x, q in zip(outs, (big, small), (qb, qsm)):
        wi, wd = oknn.knn(x, q, 1)
        assert np.array_equal(gi.cpu().numpy(), wi)
        assert np.allclose(gd.cpu().numpy(), wd, rtol=1e-5, atol=0)
    assert stats[0]["dense_queries"] >= 1
    ib.free()
    isml.free()
