"""Parity at the benchmark workloads' full sizes, in their launch
configurations: sampled queries against the FP64 oracle one by one, and for all
queries the properties that hold at any size (two independent exact engines
return the same ids; the true top-k is among the vectors the scan carried
through all dimensions)."""
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


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_exact_1m_d768_all_queries(P, torch):
    # 1M x 768 mixture, 1000 queries, PDX-BOND as the bench runs it
    x, q = pdx_synth.make("bond_exact_1m_d768")
    xd, qd = _dev(torch, x), _dev(torch, q)
    ix = P.pdx_build_layout(xd)
    log = torch.zeros(20_000_000, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    db, ib = P.pdx_search_exact(ix, qd, 10, opts=P.search_opts(pruner="bond", finished_log=log, finished_count=cnt))
    db2, ib2 = P.pdx_search_exact(ix, qd, 10)                     # the search without the log
    torch.cuda.synchronize()
    assert torch.equal(ib, ib2)
    ix.free()
    # 64 sampled queries against the oracle
    rows = np.random.default_rng(3).choice(q.shape[0], size=64, replace=False)
    check_topk(x, q, 10, db, ib, rows=rows)
    # every query: the unpruned tensor engine (TF32 GEMM, proven margins, FP32
    # rerank) returns the same ids, and all of them finished in the scan
    it = P.pdx_build_layout(xd, dense_rows=True)
    dt, idt = P.pdx_search_exact(it, qd, 10, pruner="none", engine="tensor")
    torch.cuda.synchronize()
    assert torch.equal(idt, ib)
    n_log = int(cnt.item())
    assert n_log <= log.numel()
    e = log[:n_log]
    key = (e >> 32) * x.shape[0] + (e & 0xffffffff)                  # query * n + id
    want = torch.arange(q.shape[0], device="cuda").unsqueeze(1) * x.shape[0] + idt
    assert bool(torch.isin(want.flatten(), key).all())
    np.testing.assert_allclose(db.cpu().numpy(), dt.cpu().numpy(), rtol=1e-5)


def test_learned_order_workload_2m_d1536_sampled(P, torch):
    # 2M x 1536 unit-norm vectors, inner product (searched as L2), PDX-BOND
    x, q = pdx_synth.make("learned_order_2m_d1536", nq=64)
    ix = P.pdx_build_layout(_dev(torch, x), metric="ip")
    d, i = P.pdx_search_exact(ix, _dev(torch, q), 10)
    torch.cuda.synchronize()
    check_topk(x, q, 10, d, i, metric="ip", rows=np.arange(16))


def test_serving_largest_collection_fp8_top100(P, torch):
    # the largest of the 64 serving collections (1.84M x 96), FP8 blocks,
    # exact top-100 through the server with graphs and the tuner
    colls = pdx_synth.serving_collections()
    c = max(colls, key=lambda c: c.n)
    x, q = pdx_synth.mixture_device(c.n, c.d, 16, c.seed)
    ix = P.pdx_build_layout(x, storage="fp8")
    srv = P.Server([ix], k=100, max_batch=64, use_graphs=True, autotune=True, pruner="bond")
    try:
        d1, i1 = srv.search(0, q[:1])
        d16, i16 = srv.search(0, q)
        torch.cuda.synchronize()
        xh, qh = x.cpu().numpy(), q.cpu().numpy()
        check_topk(xh, qh[:1], 100, d1, i1)
        check_topk(xh, qh, 100, d16, i16)
    finally:
        srv.free()
