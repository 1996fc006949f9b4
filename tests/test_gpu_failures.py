"""Failure paths, made on the host or by a wait that is allowed to run out (nothing here faults
the GPU): a caller allocator that returns NULL at the n-th request gives PARIS_ENOMEM with every
block released, and a device wait bound of 1 ns makes the tensor-core screening give up, drain
its own copies and MMAs and report PARIS_ETIMEOUT; after either, the next call is exact."""
import numpy as np
import pytest

from gpu_common import require_gpu, rw, torch
from oracle import knn as oknn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    import synth
    x = rw(120_000, 256, 77)
    src = synth.sigma_query_sources(x.shape[0], 6)
    q = np.concatenate([synth.noisy_queries(x[src], 0.1, [6, 1]), synth.noisy_queries(x[src], 2.0, [6, 2])])
    return x, q, oknn.knn(x, q, 3)


def workload(P, X, Q):
    """Build (BF16 copy included), then batched mixed-precision and plain exact 3-NN."""
    idx = P.paris_build_ex(X, 16, 256, bf16_shadow=True)
    try:
        a = P.paris_exact_knn_ex(idx, Q, 3, mode=P.PARIS_MODE_BATCHED, precision=P.PARIS_REFINE_MIXED,
                                 want_stats=True)
        b = P.paris_exact_knn_ex(idx, Q, 3, mode=P.PARIS_MODE_PLAIN)
        torch.cuda.synchronize()
        return a, b
    finally:
        idx.free()


def test_allocator_failure_is_enomem_and_releases_everything(data):
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x, q, (wi, wd) = data
    X, Q = torch.from_numpy(x).to(dev), torch.from_numpy(q).to(dev)
    live = {}
    state = {"n": 0, "fail_at": None}

    def alloc(nbytes, stream, _ctx):
        state["n"] += 1
        if state["fail_at"] is not None and state["n"] >= state["fail_at"]:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), dev.index or 0, stream or 0)
        live[p] = nbytes
        return p

    def free(ptr, _nbytes, _stream, _ctx):
        assert ptr in live, "freed a block the allocator did not hand out"
        del live[ptr]
        torch.cuda.caching_allocator_delete(ptr)

    P.paris_set_allocator(alloc, free)
    try:
        workload(P, X, Q)                       # first call: also tunes the query tile
        state["n"] = 0
        workload(P, X, Q)
        total = state["n"]
        assert total > 10 and not live
        for f in sorted({1, 2, 3, 5, total // 3, total // 2, total - 1, total}):
            state["n"], state["fail_at"] = 0, f
            with pytest.raises(P.ParisError) as e:
                workload(P, X, Q)
            assert e.value.status == 2, (f, str(e.value))     # PARIS_ENOMEM
            torch.cuda.synchronize()
            assert not live, (f, len(live))
        state["fail_at"] = None
        (ai, ad, _), (bi, bd) = workload(P, X, Q)
    finally:
        P.paris_set_allocator(None, None)
    for gi, gd in ((ai, ad), (bi, bd)):
        assert np.array_equal(gi.cpu().numpy(), wi)
        assert np.allclose(gd.cpu().numpy(), wd, rtol=1e-5, atol=0)


def test_expired_device_wait_is_etimeout_and_device_stays_usable(data):
    import paper_2009_00166_gb300 as P
    dev = require_gpu()
    x, q, (wi, wd) = data
    X, Q = torch.from_numpy(x).to(dev), torch.from_numpy(q).to(dev)
    idx = P.paris_build_ex(X, 16, 256, bf16_shadow=True)
    try:
        _, _, st = P.paris_exact_knn_ex(idx, Q, 3, mode=P.PARIS_MODE_BATCHED, precision=P.PARIS_REFINE_MIXED,
                                        want_stats=True)
        assert st["dense_queries"] >= 1                          # the screening runs for these queries
        P.paris_set_wait_limit(1)
        try:
            with pytest.raises(P.ParisError) as e:
                P.paris_exact_knn_ex(idx, Q, 3, mode=P.PARIS_MODE_BATCHED, precision=P.PARIS_REFINE_MIXED)
            assert e.value.status == 4                            # PARIS_ETIMEOUT
        finally:
            P.paris_set_wait_limit(0)
        with pytest.raises(P.ParisError):
            P.paris_set_wait_limit(61 * 10 ** 9)
        gi, gd = P.paris_exact_knn_ex(idx, Q, 3, mode=P.PARIS_MODE_BATCHED, precision=P.PARIS_REFINE_MIXED)
        torch.cuda.synchronize()
        assert np.array_equal(gi.cpu().numpy(), wi)
        assert np.allclose(gd.cpu().numpy(), wd, rtol=1e-5, atol=0)
    finally:
        idx.free()
