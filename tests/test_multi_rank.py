"""Multi-rank host logic on CPU gloo ranks (world size 2): job throughput aggregation (max time,
summed units) and the k-best merge of row-range shards, whose merged answer must equal the
oracle on the whole collection."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        from oracle import knn as oknn
        from paper_2009_00166_gb300 import shards
        import synth
        rate, slow = shards.job_throughput(100.0 + 50.0 * rank, 1000.0)
        x = synth.random_walk(3000, 64, seed=12)
        queries = synth.random_walk(5, 64, seed=13)
        half = x.shape[0] // world
        lo, hi = rank * half, (rank + 1) * half if rank < world - 1 else x.shape[0]
        i_loc, d_loc = oknn.knn(x[lo:hi], queries, 4)              # the per-shard exact search
        d, i = shards.merge_topk(torch.from_numpy(d_loc.astype(np.float32)), torch.from_numpy(i_loc), lo, 4)
        want_i, _ = oknn.knn(x, queries, 4)
        q.put((rank, rate, slow, bool(np.array_equal(i.numpy(), want_i))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, slow, ok in res:
        assert slow == 150.0
        assert abs(rate - 2000.0 / 0.150) < 1e-6
        assert ok
