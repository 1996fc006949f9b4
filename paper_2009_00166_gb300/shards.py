"""Host-side logic of the multi-GPU forms (one process per GPU, torch.distributed).

The search shards by rows: every rank holds a contiguous row range [offset, offset + n_local) of
one collection, builds its own index of it (no communication), and answers the same queries
over its rows; the ranks' k best (distance, row) lists are then merged into the global k best.

* ``merge_topk_exact`` orders the merged candidates by their exact distance, then by row (the
  exact search's order). The library's fp32 distances are the correctly ordered roundings of
  the exact distances, so candidates in different order positions are already ordered right;
  only candidates whose fp32 distances are EQUAL may be out of order, and those are re-ranked
  on the exact squared distance, computed in integer arithmetic by the rank that holds the row.
* ``ShardedIndex`` wraps one rank's shard: build, exact k-NN, merge.
* ``job_throughput`` sums the ranks' units over the slowest rank's time (the job's rate).
"""
from __future__ import annotations

import numpy as np


def job_throughput(local_ms: float, local_units: float, group=None):
    """(units per second of the whole job, slowest rank's ms) over all ranks of ``group``."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return local_units / (local_ms * 1e-3), local_ms
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()) / (float(t.item()) * 1e-3), float(t.item())


def _fixed(v: float) -> int:
    """An fp32 value as the exact integer v * 2^149 (every fp32 value is a multiple of 2^-149)."""
    num, den = float(v).as_integer_ratio()
    return num * ((1 << 149) // den)


def exact_sq_scaled(x_row, q_row) -> int:
    """Exact squared Euclidean distance of two fp32 vectors, as an integer multiple of 2^-298."""
    tot = 0
    for a, b in zip(np.asarray(x_row, np.float32).tolist(), np.asarray(q_row, np.float32).tolist()):
        d = _fixed(a) - _fixed(b)
        tot += d * d
    return tot


def merge_topk_exact(dist_local, idx_local, row_offset: int, k: int, queries, local_row, group=None):
    """Merge per-shard k-NN results into the global k best, ordered by (exact distance, row).

    dist_local [nq][k] fp32 and idx_local [nq][k] (rows local to the shard; -1 = no row, with
    distance +inf) are this rank's results; ``queries`` [nq][len] fp32 (host) are the queries;
    ``local_row(r)`` returns the fp32 values of local row r. Returns (dist, idx) [nq][k] with
    global rows, on every rank.
    """
    import torch
    import torch.distributed as dist
    d_loc = torch.as_tensor(dist_local, dtype=torch.float32).cpu()
    i_loc = torch.as_tensor(idx_local).to(torch.int64).cpu()
    g_loc = torch.where(i_loc >= 0, i_loc + row_offset, torch.full_like(i_loc, -1))
    if not dist.is_available() or not dist.is_initialized():
        return d_loc[:, :k].contiguous(), g_loc[:, :k].contiguous()
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    ds = [torch.empty_like(d_loc, device=dev) for _ in range(world)]
    ix = [torch.empty_like(g_loc, device=dev) for _ in range(world)]
    dist.all_gather(ds, d_loc.to(dev).contiguous(), group=group)
    dist.all_gather(ix, g_loc.to(dev).contiguous(), group=group)
    D = torch.cat([t.cpu() for t in ds], dim=1).numpy()
    I = torch.cat([t.cpu() for t in ix], dim=1).numpy()
    owner = np.repeat(np.arange(world), d_loc.shape[1])
    nq, m = D.shape
    # order by (fp32 distance, row); unused slots (row -1, +inf) sort last
    key_row = np.where(I < 0, np.iinfo(np.int64).max, I)
    order = np.lexsort((key_row, D), axis=1)
    # equal fp32 distances from different ranks among the first k: exact re-rank needed
    need = []  # (query, candidate column)
    for qi in range(nq):
        o = order[qi]
        dq = D[qi, o]
        j = 0
        while j < min(k, m):
            e = j
            while e + 1 < m and dq[e + 1] == dq[j] and np.isfinite(dq[j]):
                e += 1
            if e > j and len(set(owner[o[j:e + 1]].tolist())) > 1:
                need.extend((qi, int(c)) for c in o[j:e + 1])
            j = e + 1
    exact_mine = {}
    qh = np.asarray(queries, np.float32)
    for qi, c in need:
        if owner[c] == rank:
            exact_mine[(qi, int(I[qi, c]))] = exact_sq_scaled(local_row(int(I[qi, c]) - row_offset), qh[qi])
    gathered = [None] * world
    dist.all_gather_object(gathered, exact_mine, group=group)
    exact = {}
    for part in gathered:
        exact.update(part)
    out_d = np.empty((nq, k), np.float32)
    out_i = np.empty((nq, k), np.int64)
    for qi in range(nq):
        o = list(order[qi])
        if any(q == qi for q, _ in need):
            def rank_key(c, qi=qi):
                r = int(I[qi, c])
                return (float(D[qi, c]), exact.get((qi, r), 0), r if r >= 0 else np.iinfo(np.int64).max)
            o.sort(key=rank_key)
        out_d[qi] = D[qi, o[:k]]
        out_i[qi] = I[qi, o[:k]]
    return torch.from_numpy(out_d), torch.from_numpy(out_i)


class ShardedIndex:
    """One rank's row-range shard of a collection: rows [row_offset, row_offset + n_local)."""

    def __init__(self, series_local, row_offset: int, w: int = 16, card: int = 256, bf16_shadow: bool = False,
                 group=None):
        import paper_2009_00166_gb300 as P
        self.P = P
        self.series = series_local
        self.offset = int(row_offset)
        self.n = int(series_local.shape[0])
        self.group = group
        self.index = P.paris_build_ex(series_local, w, card, bf16_shadow=bf16_shadow)

    def exact_knn(self, queries, k: int, **query_kw):
        """Global exact k-NN of device queries over all shards: (dist [nq][k], rows [nq][k])."""
        import torch
        kk = min(k, self.n)
        i_loc, d_loc = self.P.paris_exact_knn_ex(self.index, queries, kk, **query_kw)
        if kk < k:
            pad = (queries.shape[0], k - kk)
            i_loc = torch.cat([i_loc, torch.full(pad, -1, dtype=i_loc.dtype, device=i_loc.device)], dim=1)
            d_loc = torch.cat([d_loc, torch.full(pad, float("inf"), dtype=d_loc.dtype, device=d_loc.device)], dim=1)
        qh = queries.cpu().numpy()
        series = self.series

        def local_row(r):
            return series[r].cpu().numpy()

        return merge_topk_exact(d_loc, i_loc, self.offset, k, qh, local_row, self.group)

    def free(self):
        if self.index is not None:
            self.index.free()
            self.index = None
