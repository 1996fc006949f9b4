"""Host-side logic of the multi-GPU forms (one process per GPU, torch.distributed).

* Independent problems (what ``bench.py --gpus N`` runs): every rank searches its own collection
  with its own queries; the job's throughput is the sum of the ranks' units over the slowest
  rank's time -- ``job_throughput``.
* Row-range shards of one collection: every rank answers the same queries over rows
  [offset, offset + n_local); ``merge_topk`` combines the ranks' k best (distance, row) lists,
  ordered by (distance, row). The ranks return fp32 distances, so rows whose distances from
  different shards agree to fp32 resolution are ordered by row.
"""
from __future__ import annotations


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


def merge_topk(dist_local, idx_local, row_offset: int, k: int, group=None):
    """Merge per-shard k-NN results into the global k best.

    dist_local, idx_local: [nq][k] tensors of this rank (rows local to the shard).
    Returns (dist [nq][k], idx [nq][k] global rows) on every rank.
    """
    import torch
    import torch.distributed as dist
    g_idx = idx_local.to(torch.int64) + row_offset
    if not dist.is_available() or not dist.is_initialized():
        return dist_local, g_idx
    world = dist.get_world_size(group)
    ds = [torch.empty_like(dist_local) for _ in range(world)]
    ix = [torch.empty_like(g_idx) for _ in range(world)]
    dist.all_gather(ds, dist_local.contiguous(), group=group)
    dist.all_gather(ix, g_idx.contiguous(), group=group)
    D = torch.cat(ds, dim=1)
    I = torch.cat(ix, dim=1)
    # order by (distance, row): stable sort by row, then stable sort by distance
    o1 = torch.argsort(I, dim=1, stable=True)
    D, I = torch.gather(D, 1, o1), torch.gather(I, 1, o1)
    o2 = torch.argsort(D, dim=1, stable=True)
    D, I = torch.gather(D, 1, o2), torch.gather(I, 1, o2)
    return D[:, :k].contiguous(), I[:, :k].contiguous()
