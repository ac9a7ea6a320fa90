"""GPU parity of the tensor-core dense engine (unpruned exact search as a TF32
tcgen05 GEMM with proven error margins and an FP32 rerank) against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

import pdx_synth
from oracle import knn as ok
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


def _search(P, torch, ix, q, k, engine="tensor", **kw):
    d, i, st = P.pdx_search_exact(ix, _dev(torch, q), k, pruner="none", engine=engine, stats=True, **kw)
    torch.cuda.synchronize()
    return d.cpu().numpy(), i.cpu().numpy(), st


def test_plain_config_10k_d128_tensor(P, torch):
    # the 10k x 128, 100-query, k=10 L2 workload; the tensor engine must equal
    # the oracle and, bit for bit, the PDX scan engine
    x, q = pdx_synth.make("plain_scan_10k_d128")
    ix = P.pdx_build_layout(_dev(torch, x), dense_rows=True)
    d, i, st = _search(P, torch, ix, q, 10)
    check_topk(x, q, 10, d, i)
    assert st["dense_fallbacks"] == 0
    assert st["values_visited"] == q.shape[0] * x.shape[0] * x.shape[1]
    # candidates: a small fraction of the collection is reranked
    assert 10 * q.shape[0] <= st["candidates"] < 0.2 * q.shape[0] * x.shape[0]
    ds, is_, _ = _search(P, torch, ix, q, 10, engine="scan")
    assert np.array_equal(i, is_)
    assert np.array_equal(d, ds)


@pytest.mark.parametrize("n,d,nq,k", [(1037, 128, 200, 10), (300, 36, 129, 5), (5000, 100, 1, 16),
                                      (777, 4, 7, 3), (2049, 260, 64, 64), (5, 32, 3, 10)])
def test_ragged_shapes(P, torch, n, d, nq, k):
    # vector and query counts off the 256 / 128 tile grid, d off the 32-wide
    # K chunk (zero fill), k up to 64, fewer vectors than k
    rng = np.random.default_rng(n + d)
    x = rng.standard_normal((n, d)).astype(np.float32)
    q = rng.standard_normal((nq, d)).astype(np.float32)
    ix = P.pdx_build_layout(_dev(torch, x), dense_rows=True, partition_size=1000)
    dd, ii, st = _search(P, torch, ix, q, k)
    check_topk(x, q, k, dd, ii)
    assert st["dense_fallbacks"] == 0


def test_inner_product(P, torch):
    rng = np.random.default_rng(5)
    x = (rng.standard_normal((3000, 64)) * rng.uniform(0.1, 3.0, (3000, 1))).astype(np.float32)
    q = rng.standard_normal((50, 64)).astype(np.float32)
    ix = P.pdx_build_layout(_dev(torch, x), metric="ip", dense_rows=True)
    d, i, st = _search(P, torch, ix, q, 10)
    check_topk(x, q, 10, d, i, metric="ip")
    ds, is_, _ = _search(P, torch, ix, q, 10, engine="scan")
    assert np.array_equal(i, is_) and np.array_equal(d, ds)


def test_near_ties_need_the_margin(P, torch):
    # distances that differ by ~1e-5 relative, far below TF32's resolution
    # (~1e-3): the GEMM alone cannot order them, the margin + FP32 rerank must
    rng = np.random.default_rng(11)
    d = 128
    c = rng.standard_normal(d).astype(np.float32)
    x = (c + 1e-3 * rng.standard_normal((4000, d))).astype(np.float32)
    x[::7] = (rng.standard_normal((len(x[::7]), d))).astype(np.float32)
    q = (c + 0.3 * rng.standard_normal((40, d))).astype(np.float32)
    ix = P.pdx_build_layout(_dev(torch, x), dense_rows=True)
    dd, ii, st = _search(P, torch, ix, q, 10)
    check_topk(x, q, 10, dd, ii)
    # the scan engine picks its k from scan-order FP32 sums before the
    # canonical rerank, so on ties this close the engines may differ, each
    # within the tie tolerance
    ds, is_, _ = _search(P, torch, ix, q, 10, engine="scan")
    check_topk(x, q, 10, ds, is_)


def test_wide_dynamic_range(P, torch):
    rng = np.random.default_rng(12)
    x = rng.standard_normal((3000, 96)).astype(np.float32)
    x *= np.float32(10.0) ** rng.integers(-3, 4, size=(3000, 1)).astype(np.float32)
    q = rng.standard_normal((30, 96)).astype(np.float32) * np.float32(5.0)
    ix = P.pdx_build_layout(_dev(torch, x), dense_rows=True)
    dd, ii, st = _search(P, torch, ix, q, 10)
    check_topk(x, q, 10, dd, ii)


def test_duplicates_overflow_to_exact_fallback(P, torch):
    # 6000 copies of the same vector nearest to every query: all fall inside
    # the margin band, the candidate buffer overflows, and the finish kernel
    # answers by a plain FP32 scan; ties go to the lower ids
    rng = np.random.default_rng(13)
    d = 64
    x = rng.standard_normal((9000, d)).astype(np.float32) * 3
    base = rng.standard_normal(d).astype(np.float32)
    x[1000:7000] = base
    q = (base + 0.01 * rng.standard_normal((4, d))).astype(np.float32)
    ix = P.pdx_build_layout(_dev(torch, x), dense_rows=True)
    dd, ii, st = _search(P, torch, ix, q, 10)
    assert st["dense_fallbacks"] == 4
    check_topk(x, q, 10, dd, ii)
    assert (ii == np.arange(1000, 1010)[None, :]).all()


def test_low_precision_index_uses_fp32_rows(P, torch):
    rng = np.random.default_rng(14)
    x = rng.standard_normal((2500, 128)).astype(np.float32)
    q = rng.standard_normal((20, 128)).astype(np.float32)
    ix = P.pdx_build_layout(_dev(torch, x), storage="fp8", dense_rows=True)
    dd, ii, st = _search(P, torch, ix, q, 10)
    check_topk(x, q, 10, dd, ii)


def test_engine_selection_and_errors(P, torch):
    rng = np.random.default_rng(15)
    x = rng.standard_normal((500, 30)).astype(np.float32)
    q = rng.standard_normal((4, 30)).astype(np.float32)
    plain = P.pdx_build_layout(_dev(torch, x[:, :28]))            # no row-major copy
    odd = P.pdx_build_layout(_dev(torch, x), dense_rows=True)      # d % 4 != 0
    for ix in (plain, odd):
        with pytest.raises(P.PdxError, match="UNSUPPORTED"):
            P.pdx_search_exact(ix, _dev(torch, q[:, :ix.info.d]), 5, pruner="none", engine="tensor")
        # AUTO quietly takes the scan engine
        d, i = P.pdx_search_exact(ix, _dev(torch, q[:, :ix.info.d]), 5, pruner="none")
        check_topk(x[:, :ix.info.d], q[:, :ix.info.d], 5, d, i)
    dense = P.pdx_build_layout(_dev(torch, x[:, :28]), dense_rows=True)
    with pytest.raises(P.PdxError, match="UNSUPPORTED"):
        P.pdx_search_exact(dense, _dev(torch, q[:, :28]), 5, pruner="bond", engine="tensor")
    with pytest.raises(P.PdxError, match="UNSUPPORTED"):
        P.pdx_search_exact(dense, _dev(torch, q[:, :28]), 65, pruner="none", engine="tensor")
    # host query and output pointers take the same path
    d, i = P.pdx_search_exact(dense, q[:, :28], 5, pruner="none", engine="tensor")
    check_topk(x[:, :28], q[:, :28], 5, d, i)


def test_noalloc_entry_takes_the_tensor_engine(P, torch):
    x, q = pdx_synth.make("plain_scan_10k_d128")
    ix = P.pdx_build_layout(_dev(torch, x), dense_rows=True)
    d, i = P.pdx_search_exact_noalloc(ix, _dev(torch, q), 10, pruner="none", engine="tensor")
    torch.cuda.synchronize()
    check_topk(x, q, 10, d, i)


def test_full_size_1m_d768_sampled(P, torch):
    # the 1M x 768 mixture with its 1000 queries, unpruned on the tensor
    # engine; the oracle checks a sample of the queries one by one
    x, q = pdx_synth.make("bond_exact_1m_d768")
    ix = P.pdx_build_layout(_dev(torch, x), dense_rows=True)
    d, i, st = _search(P, torch, ix, q, 10)
    assert st["dense_fallbacks"] == 0
    rows = np.random.default_rng(2).choice(q.shape[0], size=6, replace=False)
    check_topk(x, q, 10, d, i, rows=rows)


def test_gemm_wait_timeout_is_reported_and_answered(P, torch, monkeypatch):
    # test hook: the GEMM's producer loads nothing, so its MMA thread's first
    # wait runs out after its 2 s limit. The kernel releases TMEM and flags the
    # error; the finish kernel then answers every query by the plain FP32 scan.
    # No fault is involved, and the context stays usable.
    rng = np.random.default_rng(16)
    x = rng.standard_normal((3000, 64)).astype(np.float32)
    q = rng.standard_normal((8, 64)).astype(np.float32)
    ix = P.pdx_build_layout(_dev(torch, x), dense_rows=True)
    monkeypatch.setenv("PDX_TEST_DENSE_STALL", "1")
    d, i, st = _search(P, torch, ix, q, 10)
    assert st["dense_fallbacks"] == q.shape[0]
    check_topk(x, q, 10, d, i)
    monkeypatch.delenv("PDX_TEST_DENSE_STALL")
    d, i, st = _search(P, torch, ix, q, 10)
    assert st["dense_fallbacks"] == 0
    check_topk(x, q, 10, d, i)
