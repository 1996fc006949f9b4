"""Row-range shards of one collection through the library: two gloo ranks (processes) each build
the index of half the rows on cuda:0 and answer the same queries; the exact merge must return
the oracle's answer over the whole collection, including a planted cross-shard pair whose
distances round to the same fp32 value. The ranks' kernels never wait on one another; only the
host-side gloo collectives connect them."""
import os

import numpy as np
import pytest

from gpu_common import require_gpu, torch

pytestmark = pytest.mark.gpu


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        sys.path.insert(0, root)
        sys.path.insert(0, os.path.join(root, "tests"))
        import torch as T
        from paper_2009_00166_gb300 import shards
        from test_multi_rank import planted_collection
        T.cuda.set_device(0)
        x, q = planted_collection()
        half = x.shape[0] // world
        lo, hi = rank * half, (rank + 1) * half if rank < world - 1 else x.shape[0]
        sh = shards.ShardedIndex(T.from_numpy(x[lo:hi]).cuda(), lo)
        res = []
        for k in (1, 3):
            for mode in (0, 1):
                d, i = sh.exact_knn(T.from_numpy(q).cuda(), k, mode=mode)
                res.append((k, i.numpy(), d.numpy()))
        sh.free()
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_sharded_search_two_ranks():
    import torch.multiprocessing as mp
    from oracle import knn as oknn
    from test_multi_rank import planted_collection
    require_gpu()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 31000 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = [out.get(timeout=600) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    x, q = planted_collection()
    for _, rs in res:
        for k, gi, gd in rs:
            wi, wd = oknn.knn(x, q, k)
            assert np.array_equal(gi, wi)
            assert np.allclose(gd, wd, rtol=1e-5, atol=0)
            assert gi[0, 0] == 2000
