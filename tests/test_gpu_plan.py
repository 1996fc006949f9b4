"""Captured batches (paris_knn_plan_*): the first run executes eagerly and records the call as
a CUDA graph; later runs replay it. Every run's answers equal the oracle's and the eager call's,
for both refinement precisions, k in {1, 10}, plain and batched scans, several chunks per
batch, host or device buffers, and a batch whose tensor-core screening overflows a list (the
run is redone eagerly with the repeated screenings)."""
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
    batches = [synth.mixed_sigma_queries(x, x.shape[0], 256, 21, 0.01, 2.0, seed=60 + b)[0] for b in range(3)]
    want = {k: [oknn.knn(x, q, k) for q in batches] for k in (1, 10)}
    yield P, idx, batches, want
    idx.free()


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("k", [1, 10])
@pytest.mark.parametrize("mode,chunk", [("batched", 0), ("batched", 5), ("plain", 0)])
def test_plan_replays_match_oracle(setup, precision, k, mode, chunk):
    P, idx, batches, want = setup
    prec = P.PARIS_REFINE_FP32 if precision == "fp32" else P.PARIS_REFINE_MIXED
    md = P.PARIS_MODE_BATCHED if mode == "batched" else P.PARIS_MODE_PLAIN
    plan = P.KnnPlan(idx, 21, k, mode=md, chunk=chunk, precision=prec)
    for rep in range(2):
        for b, q in enumerate(batches):
            gi, gd = plan.run(torch.from_numpy(q).cuda())
            wi, wd = want[k][b]
            assert np.array_equal(gi.cpu().numpy(), wi), (rep, b)
            assert np.allclose(gd.cpu().numpy(), wd, rtol=1e-5, atol=0), (rep, b)
    info = plan.info()
    assert info["captured"] == 1 and info["graph_kernels"] > 0
    assert info["eager_runs"] == 1 and info["replays"] == 5
    eager = P.paris_exact_knn_ex(idx, torch.from_numpy(batches[0]).cuda(), k, mode=md, chunk=chunk, precision=prec)
    again = plan.run(torch.from_numpy(batches[0]).cuda())
    assert np.array_equal(eager[0].cpu().numpy(), again[0].cpu().numpy())
    assert np.array_equal(eager[1].cpu().numpy(), again[1].cpu().numpy())
    plan.free()


def test_plan_host_buffers(setup):
    P, idx, batches, want = setup
    plan = P.KnnPlan(idx, 21, 1, precision=P.PARIS_REFINE_MIXED)
    for b in (0, 1, 2, 0):
        oi = np.empty((21, 1), np.int64)
        od = np.empty((21, 1), np.float32)
        plan.run(batches[b], oi, od)                     # host queries and outputs
        assert np.array_equal(oi, want[1][b][0])
        assert np.allclose(od, want[1][b][1], rtol=1e-5, atol=0)
    assert plan.info()["replays"] == 3
    plan.free()


def test_plan_overflowed_screening_runs_eagerly():
    """Loose queries whose tensor-core candidate lists overflow at k = 16: the replay notices the
    overflow and the run is redone eagerly, with the same exact answers."""
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    n = 300_007
    x = synth.random_walk(n, 256, seed=9)
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    src = np.random.default_rng(4).choice(n, 24, replace=False)
    q = synth.noisy_queries(x[src], 2.0, [5, 1])
    wi, wd = oknn.knn(x, q, 16)
    _, _, st = P.paris_exact_knn_ex(idx, torch.from_numpy(q).cuda(), 16, mode=P.PARIS_MODE_BATCHED,
                                    precision=P.PARIS_REFINE_MIXED, want_stats=True)
    plan = P.KnnPlan(idx, 24, 16, precision=P.PARIS_REFINE_MIXED)
    for _ in range(3):
        gi, gd = plan.run(torch.from_numpy(q).cuda())
        assert np.array_equal(gi.cpu().numpy(), wi)
        assert np.allclose(gd.cpu().numpy(), wd, rtol=1e-5, atol=0)
    info = plan.info()
    assert info["captured"] == 1
    if st["rescreens"] > 0:                              # every replay fell back to the eager run
        assert info["eager_runs"] == 3 and info["replays"] == 2
    plan.free()
    idx.free()


def test_plan_rejects_bad_arguments(setup):
    P, idx, batches, _ = setup
    with pytest.raises(P.ParisError):
        P.KnnPlan(idx, 0, 1)
    with pytest.raises(P.ParisError):
        P.KnnPlan(idx, 4, 0)


def test_multi_collection_plan_replays_match_oracle():
    """Three collections of lengths 128, 256 and 1024 (uneven query counts, one collection with
    no queries in the second plan) recorded as one graph: every replay equals the oracle and the
    eager multi-collection call."""
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    shapes = [(60_000, 128, 41), (40_000, 256, 42), (6_000, 1024, 43)]
    xs = [synth.random_walk(n, length, seed=s) for n, length, s in shapes]
    idxs = [P.paris_build_ex(torch.from_numpy(x).to(dev), bf16_shadow=x.shape[1] <= 256) for x in xs]
    for nqs in ([9, 14, 5], [12, 0, 7]):
        for prec in (P.PARIS_REFINE_FP32, P.PARIS_REFINE_MIXED):
            plan = P.KnnPlanMulti(idxs, nqs, 3, precision=prec)
            for rep in range(3):
                qs = [synth.mixed_sigma_queries(x, x.shape[0], x.shape[1], m, 0.01, 2.0, seed=70 + 10 * rep + c)[0]
                      if m else np.zeros((0, x.shape[1]), np.float32) for c, (x, m) in enumerate(zip(xs, nqs))]
                Qs = [torch.from_numpy(np.ascontiguousarray(q)).to(dev) for q in qs]
                outs = plan.run(Qs)
                eager = P.paris_exact_knn_multi(idxs, Qs, 3, precision=prec)
                for c, (x, q) in enumerate(zip(xs, qs)):
                    if not len(q):
                        continue
                    wi, wd = oknn.knn(x, q, 3)
                    gi, gd = outs[c][0].cpu().numpy(), outs[c][1].cpu().numpy()
                    assert np.array_equal(gi, wi), (nqs, prec, rep, c)
                    assert np.allclose(gd, wd, rtol=1e-5, atol=0)
                    assert np.array_equal(gi, eager[c][0].cpu().numpy())
            info = plan.info()
            assert info["captured"] == 1 and info["replays"] + info["eager_runs"] == 3 and info["replays"] >= 1
            plan.free()
    with pytest.raises(P.ParisError):
        P.KnnPlanMulti(idxs, [0, 0, 0], 3)
    for ix in idxs:
        ix.free()
