"""Low-precision PDX storage (BF16 / FP8-E4M3 with per-dimension scales): the
stored codes equal the oracle's rounding bit for bit, and searches stay exact
against the FP64 oracle on the FP32 data. PDX-BOND prunes on a lower bound
widened by the per-element quantisation bound, and survivors are reranked in
FP32."""
import numpy as np
import pytest

import pdx_synth
from oracle import knn as ok
from oracle import quant as Q
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


def _expected_blocks(x, ps):
    n, d = x.shape
    nparts = -(-n // ps)
    size = -(-n // nparts)
    blocks = []
    for p in range(nparts):
        rows = np.arange(p * size, min(n, (p + 1) * size))
        for t in range(0, rows.size, 64):
            sl = rows[t:t + 64]
            b = np.zeros((d, 64), np.float32)
            b[:, :sl.size] = x[sl].T
            blocks.append(b)
    return np.stack(blocks)


def test_stored_codes_match_oracle_rounding(P, torch):
    rng = np.random.default_rng(0)
    x = (rng.standard_normal((700, 40)) * rng.uniform(0.001, 50, 40)).astype(np.float32)
    exp = _expected_blocks(x, 300)
    ib = P.pdx_build_layout(_dev(torch, x), partition_size=300, storage="bf16")
    got = ib.copy_out("blocks_lp")
    want = (Q.bf16_round(exp).view(np.uint32) >> 16).astype(np.uint16)
    assert np.array_equal(got, want)
    i8 = P.pdx_build_layout(_dev(torch, x), partition_size=300, storage="fp8")
    sc = i8.copy_out("scales")
    want_s = (np.abs(x).max(axis=0) / np.float32(448.0)).astype(np.float32)
    assert np.array_equal(sc, want_s)
    codes = i8.copy_out("blocks_lp")
    dec = Q.e4m3_values()[codes]
    ref = Q.e4m3_round((exp / sc[None, :, None]).astype(np.float32).astype(np.float64))
    assert np.array_equal(dec, ref)


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
@pytest.mark.parametrize("pruner", ["none", "bond"])
@pytest.mark.parametrize("n,d,k,ps", [(1000, 37, 10, 300), (3000, 96, 33, 1000), (5, 3, 10, 10000)])
def test_exact_search_low_precision(P, torch, storage, pruner, n, d, k, ps):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=n, d=d, nq=13, n_centres=7, seed=n + d + 1))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=ps, storage=storage)
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), k, pruner=pruner)
    torch.cuda.synchronize()
    check_topk(x, q, k, dist, idx, atol=1e-5)


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_low_precision_mixture_768(P, torch, storage):
    x, q = pdx_synth.make("bond_exact_1m_d768", n=60_000, nq=24)
    ix = P.pdx_build_layout(_dev(torch, x), storage=storage)
    ref = P.pdx_build_layout(_dev(torch, x))
    d, i, st = P.pdx_search_exact(ix, _dev(torch, q), 10, stats=True)
    _, _, sf = P.pdx_search_exact(ref, _dev(torch, q), 10, stats=True)
    torch.cuda.synchronize()
    check_topk(x, q, 10, d, i)
    esize = 2 if storage == "bf16" else 1
    assert st["bytes_logical"] < sf["bytes_logical"]
    # the margin costs some pruning, but not most of it
    assert st["values_visited"] < 3 * sf["values_visited"]
    assert st["vectors_pruned"] > 0.9 * sf["vectors_pruned"]
    del esize


def test_low_precision_ivf_and_unit_ip(P, torch):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=6000, d=48, nq=24, n_centres=24, seed=41))
    init = np.ascontiguousarray(x[np.random.default_rng(41).choice(6000, size=24, replace=False)])
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=24, kmeans_iters=0, init_centroids=init, storage="bf16")
    oa, _ = ok.assign(x, init)
    truth = ok.knn_probed(x, q, 10, oa, init, 5)
    dist, idx = P.pdx_search_ivf(ix, _dev(torch, q), 10, 5, pruner="bond")
    torch.cuda.synchronize()
    c = init.astype(np.float64)
    rows = [r for r in range(24)
            if (lambda dd: dd[5] - dd[4] > 1e-4 * dd[5])(np.sort(((c - q[r]) ** 2).sum(axis=1)))]
    rows = np.array(rows)
    check_topk(x, q, 10, dist, idx, truth=(truth[0][rows], truth[1][rows]), rows=rows)
    xu, qu = pdx_synth.embedding_like(3000, 64, 9, n_clusters=16, rank=8)
    iu = P.pdx_build_layout(_dev(torch, xu), metric="ip", storage="fp8", partition_size=1000)
    dist, idx = P.pdx_search_exact(iu, _dev(torch, qu), 10)
    torch.cuda.synchronize()
    check_topk(xu, qu, 10, dist, idx, metric="ip", atol=2e-6)


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_low_precision_k100_d1024(P, torch, storage):
    # the serving workload's shape: exact top-100 over 1024-dimensional
    # low-precision blocks (margin-widened lower bound, FP32 rerank)
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=20000, d=1024, nq=24, n_centres=16, seed=44))
    ix = P.pdx_build_layout(_dev(torch, x), storage=storage)
    for pruner in ("none", "bond"):
        dist, idx = P.pdx_search_exact(ix, _dev(torch, q), 100, pruner=pruner)
        torch.cuda.synchronize()
        check_topk(x, q, 100, dist, idx)
