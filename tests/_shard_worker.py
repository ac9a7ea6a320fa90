"""Rank body of the sharded-search test: one CPU process per rank, gloo
collectives. Each rank answers the queries over its own id range of the
collection with the FP64 oracle (standing in for that rank's GPU search),
makes its ids global, all-gathers the per-shard lists and merges them with
the library's pdx_merge_topk (host path)."""
import os

import numpy as np


def rank_main(rank, world, port, x, q, k, metric, out_path):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import knn as ok
        from paper_2503_04422_gb300 import pdx

        n = x.shape[0]
        lo, hi = rank * n // world, (rank + 1) * n // world
        d_, i_ = ok.knn(x[lo:hi], q, k, metric)
        i_ = np.where(i_ >= 0, i_ + lo, -1).astype(np.int64)
        dt = torch.from_numpy(d_.astype(np.float32))
        it = torch.from_numpy(i_)
        gd = [torch.empty_like(dt) for _ in range(world)]
        gi = [torch.empty_like(it) for _ in range(world)]
        dist.all_gather(gd, dt)
        dist.all_gather(gi, it)
        md, mi = pdx.pdx_merge_topk(torch.stack(gd).numpy(), torch.stack(gi).numpy(), metric)
        # every rank holds the same merged answer
        chk = torch.from_numpy(mi.copy())
        ref = chk.clone()
        dist.broadcast(ref, src=0)
        assert torch.equal(chk, ref)
        if rank == 0:
            np.savez(out_path, d=md, i=mi)
        dist.barrier()
    finally:
        dist.destroy_process_group()
