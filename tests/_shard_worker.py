"""Rank body of the sharded-search test: one CPU process per rank, gloo
collectives. Each rank answers the queries over its own id range of the
collection with the FP64 oracle (standing in for that rank's GPU search),
and hands its lists to paper_2503_04422_gb300.shard.gather_merge (global
ids, all-gather, the library's pdx_merge_topk on the host path), the same
exchange step the bench's sharded mode runs over NCCL."""
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
        from paper_2503_04422_gb300 import shard

        n = x.shape[0]
        lo, hi = shard.shard_range(n, rank, world)
        d_, i_ = ok.knn(x[lo:hi], q, k, metric)
        # the bench's exchange step: global ids, all-gather, pdx_merge_topk
        md, mi = shard.gather_merge(torch.from_numpy(d_.astype(np.float32)), torch.from_numpy(i_.astype(np.int64)),
                                    lo, metric)
        md, mi = md.numpy(), mi.numpy()
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
