"""paris_lb_scan_noalloc: the lower-bound scan for callers that cannot have the library allocate
device memory while they run (services that reserve all device memory up front and forbid
allocation on the request path; hosts that pass only pre-existing buffers). Its scratch lives
in a static device array, so it must give the same kept rows and bounds as paris_lb_scan, call
after call, even though every call reuses the previous call's scratch contents.

This file is named to be collected last; it passes alone in a fresh process and after the rest.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_common import require_gpu, small_dataset, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2009_00166_gb300 as P
    import synth
    dev = require_gpu()
    x = small_dataset()
    idx = P.paris_build(torch.from_numpy(x).to(dev), 16, 256)
    src = synth.sigma_query_sources(x.shape[0], 4)
    qa = np.concatenate([synth.noisy_queries(x[src], 0.1, [4, 1]), synth.random_walk(2, 256, seed=2)])
    qb = np.concatenate([synth.noisy_queries(x[src], 1.0, [4, 2]), synth.random_walk(3, 256, seed=3)])
    yield P, idx, x, qa.astype(np.float32), qb.astype(np.float32)
    idx.free()


def noalloc(P, idx, q, thr, cap):
    L = P.lib()
    L.paris_lb_scan_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int64, C.c_void_p, C.c_void_p]
    L.paris_lb_scan_noalloc.restype = C.c_int32
    nq = q.shape[0]
    Q = torch.from_numpy(q).cuda()
    rows = torch.empty((nq, cap), dtype=torch.int32, device="cuda")
    lbs = torch.empty((nq, cap), dtype=torch.float32, device="cuda")
    th = np.ascontiguousarray(thr, dtype=np.float32)
    counts = np.zeros(nq, np.int64)
    st = L.paris_lb_scan_noalloc(idx.handle, Q.data_ptr(), nq, th.ctypes.data, rows.data_ptr(), lbs.data_ptr(), cap,
                                 counts.ctypes.data, torch.cuda.current_stream().cuda_stream)
    assert st == 0, P.paris_last_error()
    torch.cuda.synchronize()
    return rows.cpu().numpy().view(np.uint32), lbs.cpu().numpy(), counts


def thresholds(P, idx, q):
    _, seed = P.paris_approx_search(idx, torch.from_numpy(q).cuda(), 1)
    return seed.cpu().numpy() * 1.5


def test_noalloc_matches_lb_scan_twice(setup):
    P, idx, x, qa, qb = setup
    cap = x.shape[0]
    for q in (qa, qb):                                    # two calls in a row share the scratch
        thr = thresholds(P, idx, q)
        rows, lbs, counts = noalloc(P, idx, q, thr, cap)
        for t in range(q.shape[0]):
            r_ref, lb_ref, c_ref = P.paris_lb_scan(idx, torch.from_numpy(q[t]).cuda(), float(thr[t]))
            assert counts[t] == c_ref
            got = dict(zip(rows[t, :counts[t]].tolist(), lbs[t, :counts[t]].tolist()))
            want = dict(zip(r_ref.cpu().numpy().tolist(), lb_ref.cpu().numpy().tolist()))
            assert got.keys() == want.keys()
            for r, v in want.items():
                assert abs(got[r] - v) <= 1e-6 * max(v, 1e-30)


def test_noalloc_counts_only_and_limit(setup):
    P, idx, x, qa, _ = setup
    thr = thresholds(P, idx, qa)
    _, _, c0 = noalloc(P, idx, qa, thr, 0)
    _, _, c1 = noalloc(P, idx, qa, thr, x.shape[0])
    assert np.array_equal(c0, c1)
    L = P.lib()
    big = np.zeros((64, 256), np.float32)                # 64 queries at 256 symbols exceed the scratch
    Q = torch.from_numpy(big).cuda()
    counts = np.zeros(64, np.int64)
    th = np.ones(64, np.float32)
    st = L.paris_lb_scan_noalloc(idx.handle, Q.data_ptr(), 64, th.ctypes.data, None, None, 0, counts.ctypes.data,
                                 torch.cuda.current_stream().cuda_stream)
    assert st == 1 and "static scratch" in P.paris_last_error()


def test_noalloc_calls_no_allocator(setup):
    """The defining property: with a counting allocator installed (every library allocation goes
    through it), paris_lb_scan allocates and paris_lb_scan_noalloc does not."""
    P, idx, x, qa, _ = setup
    thr = thresholds(P, idx, qa)
    noalloc(P, idx, qa, thr, 16)                          # device set-up done before counting
    calls = {"alloc": 0, "free": 0}

    def alloc(nbytes, stream, _ctx):
        calls["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)

    def free(ptr, _nbytes, _stream, _ctx):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    P.paris_set_allocator(alloc, free)
    try:
        P.paris_lb_scan(idx, torch.from_numpy(qa[0]).cuda(), float(thr[0]))
        torch.cuda.synchronize()
        assert calls["alloc"] > 0                           # the counter sees the library
        calls["alloc"] = calls["free"] = 0
        for _ in range(2):
            _, _, counts = noalloc(P, idx, qa, thr, x.shape[0])
            assert counts.sum() > 0
        assert calls == {"alloc": 0, "free": 0}
    finally:
        P.paris_set_allocator(None, None)
