"""Sharded exact search across CPU ranks (world size 2, gloo): per-shard
top-k lists with global ids, all-gathered and merged by the library's
pdx_merge_topk, equal the FP64 oracle's top-k over the whole collection."""
import socket

import numpy as np
import pytest

from oracle import knn as ok
from tests._parity import check_topk


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _run(x, q, k, metric, tmp_path, world=2):
    import torch.multiprocessing as mp

    from tests._shard_worker import rank_main
    out = str(tmp_path / "merged.npz")
    mp.spawn(rank_main, args=(world, _free_port(), x, q, k, metric, out), nprocs=world, join=True)
    r = np.load(out)
    return r["d"], r["i"]


def test_integer_grid_l2_matches_whole_collection(tmp_path):
    # integer coordinates: every distance is an exact integer in FP32 and FP64,
    # so ties are real and must go to the lower global id
    rng = np.random.default_rng(3)
    x = rng.integers(-3, 4, size=(600, 6)).astype(np.float32)
    q = rng.integers(-3, 4, size=(20, 6)).astype(np.float32)
    d, i = _run(x, q, 12, "l2", tmp_path)
    td, ti = ok.knn(x, q, 12)
    assert np.array_equal(i, ti)
    assert np.array_equal(d, td.astype(np.float32))


def test_inner_product_random(tmp_path):
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1500, 32)).astype(np.float32)
    q = rng.standard_normal((16, 32)).astype(np.float32)
    d, i = _run(x, q, 10, "ip", tmp_path)
    check_topk(x, q, 10, d, i, metric="ip")


def test_shards_smaller_than_k(tmp_path):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((15, 8)).astype(np.float32)
    q = rng.standard_normal((3, 8)).astype(np.float32)
    d, i = _run(x, q, 10, "l2", tmp_path)
    check_topk(x, q, 10, d, i)


def test_merge_argument_errors():
    from paper_2503_04422_gb300 import pdx
    dist = np.zeros((2, 3, 4), np.float32)
    idx = np.zeros((2, 3, 4), np.int64)
    with pytest.raises(pdx.PdxError, match="ERR_ARG"):
        pdx.pdx_merge_topk(np.zeros((65, 1, 4), np.float32), np.zeros((65, 1, 4), np.int64))
    d, i = pdx.pdx_merge_topk(dist, idx)      # equal keys: lower id first, then the next shard's
    assert d.shape == (3, 4) and i.shape == (3, 4)
