"""Batched serving (pdx_server_*): every batch of every collection returns the
exact top-k (FP64 oracle), whether it is served by a freshly tuned entry, by
replaying its CUDA graph, or without graphs; tuning results round-trip
through the JSON cache."""
import json
import os

import numpy as np
import pytest

import pdx_synth
from tests._parity import check_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2503_04422_gb300 import build as pbuild
    pbuild.build()
    from paper_2503_04422_gb300 import pdx
    return pdx


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    return t


@pytest.fixture(scope="module")
def collections(P, torch):
    specs = [(3000, 96, "f32"), (20000, 384, "fp8"), (700, 40, "bf16")]
    out = []
    for i, (n, d, st) in enumerate(specs):
        x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=n, d=d, nq=80, n_centres=12, seed=50 + i))
        ix = P.pdx_build_layout(torch.from_numpy(x).cuda(), partition_size=4000, storage=st)
        out.append((x, q, ix))
    return out


@pytest.mark.parametrize("graphs,tune", [(True, True), (False, False), (True, False)])
def test_server_batches_are_exact(P, torch, collections, graphs, tune, tmp_path):
    cache = str(tmp_path / "tune.json")
    srv = P.Server([c[2] for c in collections], k=7, max_batch=64, use_graphs=graphs, autotune=tune,
                   tune_cache=cache if tune else None)
    rng = np.random.default_rng(1)
    stream = [(int(rng.integers(0, 3)), int(b)) for b in [1, 3, 17, 64, 5, 3, 64, 33, 1]]
    launches0 = P.pdx_kernel_launches()
    for coll, b in stream:
        x, q, _ = collections[coll]
        sel = rng.choice(q.shape[0], size=b, replace=False)
        qq = np.ascontiguousarray(q[sel])
        d, i = srv.search(coll, torch.from_numpy(qq).cuda())
        torch.cuda.synchronize()
        check_topk(x, qq, 7, d, i)
        dh, ih = srv.search(coll, qq)                 # host buffers
        assert np.array_equal(ih, i.cpu().numpy())
    info = srv.info
    # every batch runs the library's kernels, graph replays included
    assert P.pdx_kernel_launches() - launches0 >= 2 * len(stream)
    if graphs:
        assert info["graph_launches"] > 0 and info["direct_launches"] == 0
    else:
        assert info["graph_launches"] == 0
    if tune:
        assert info["tunings"] >= 1
        data = json.load(open(cache))
        assert len(data) == info["tunings"]
        # a second server reads the cache instead of tuning again
        srv2 = P.Server([c[2] for c in collections], k=7, max_batch=64, tune_cache=cache)
        x, q, _ = collections[stream[0][0]]
        d, i = srv2.search(stream[0][0], np.ascontiguousarray(q[:stream[0][1]]))
        assert srv2.info["tunings"] == 0
        check_topk(x, q[:stream[0][1]], 7, d, i)
        srv2.free()
    srv.free()


def test_server_argument_errors(P, torch, collections):
    srv = P.Server([collections[0][2]], k=5, max_batch=16, autotune=False)
    q = collections[0][1]
    with pytest.raises(P.PdxError):
        srv.search(1, q[:4])                               # no such collection
    with pytest.raises(P.PdxError):
        srv.search(0, q[:17])                              # above max_batch
    srv.free()


def test_server_fp8_top100(P, torch):
    # FP8-E4M3 storage, exact top-100 L2, graph replays and autotuning: the
    # serving configuration, checked against the FP64 oracle
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=20000, d=384, nq=96, n_centres=16, seed=57))
    ix = P.pdx_build_layout(torch.from_numpy(x).cuda(), storage="fp8")
    srv = P.Server([ix], k=100, max_batch=64, use_graphs=True, autotune=True)
    off = 0
    for b in (1, 64, 7, 24):
        qq = np.ascontiguousarray(q[off:off + b])
        off += b
        d, i = srv.search(0, torch.from_numpy(qq).cuda())
        torch.cuda.synchronize()
        check_topk(x, qq, 100, d, i)
    assert srv.info["graph_launches"] > 0
    srv.free()
