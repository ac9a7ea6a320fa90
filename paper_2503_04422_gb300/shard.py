"""Sharded search across ranks: the exchange step of a collection split over
GPUs (not in the paper, whose search runs on one machine).

Each rank holds one contiguous id range of the collection and answers the
same queries over it. The per-shard lists (distances and ids, best first) are
all-gathered with torch.distributed (NCCL for device tensors, gloo for host
tensors) and merged by the library's pdx_merge_topk, on the device for CUDA
tensors and on the calling thread for host tensors. Ids are made global first
by adding the shard's first id. Argument marshalling only: the merge runs in
libpdx.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Ids [lo, hi) of this rank's shard: equal contiguous ranges in id order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return rank * n // world, (rank + 1) * n // world


def gather_merge(dist_local, idx_local, lo: int, metric: str = "l2", group=None):
    """All ranks: (dist, idx) [nq][k] over this rank's shard (shard-local ids,
    padding -1) -> the merged [nq][k] over the whole collection (global ids),
    the same on every rank."""
    import torch
    import torch.distributed as dist

    from . import pdx

    idx_g = torch.where(idx_local >= 0, idx_local + lo, idx_local).to(torch.int64).contiguous()
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return dist_local, idx_g                      # one shard: nothing to exchange
    world = dist.get_world_size(group)
    dist_local = dist_local.contiguous()
    gd = [torch.empty_like(dist_local) for _ in range(world)]
    gi = [torch.empty_like(idx_g) for _ in range(world)]
    dist.all_gather(gd, dist_local, group=group)
    dist.all_gather(gi, idx_g, group=group)
    sd, si = torch.stack(gd), torch.stack(gi)
    if sd.is_cuda:
        return pdx.pdx_merge_topk(sd, si, metric)
    md, mi = pdx.pdx_merge_topk(sd.numpy(), si.numpy(), metric)
    return torch.from_numpy(md), torch.from_numpy(mi)
