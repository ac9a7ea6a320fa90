"""GPU parity of the exact path (layout build, PDX linear scan, PDX-BOND)
against the FP64 oracle, through the C ABI."""
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


def test_layout_matches_definition(P, torch):
    # Sec. 3: part p = rows [p*S, (p+1)*S), its blocks hold rows in order,
    # element (vector t, dim j) of block b at [(b*D + j)*64 + t], zero padding
    rng = np.random.default_rng(0)
    n, d, ps = 1000, 37, 300
    x = rng.standard_normal((n, d)).astype(np.float32)
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=ps)
    inf = ix.info
    nparts = -(-n // ps)
    size = -(-n // nparts)
    assert inf.nparts == nparts and inf.n == n and inf.d == d
    pb = ix.copy_out("part_blocks")
    ids = ix.copy_out("ids")
    blocks = ix.copy_out("blocks")
    means = ix.copy_out("means")
    b = 0
    for p in range(nparts):
        rows = np.arange(p * size, min(n, (p + 1) * size))
        nb = -(-rows.size // 64)
        assert pb[p] == b and pb[p + 1] == b + nb
        for t in range(nb):
            sl = rows[t * 64:(t + 1) * 64]
            exp_ids = np.full(64, -1, np.int32)
            exp_ids[:sl.size] = sl
            assert (ids[(b + t) * 64:(b + t + 1) * 64] == exp_ids).all()
            exp = np.zeros((d, 64), np.float32)
            exp[:, :sl.size] = x[sl].T
            assert np.array_equal(blocks[b + t], exp)
        np.testing.assert_allclose(means[p], x[rows].astype(np.float64).mean(axis=0), rtol=1e-5, atol=1e-6)
        b += nb
    assert blocks.shape[0] == b


@pytest.mark.parametrize("pruner", ["none", "bond"])
@pytest.mark.parametrize("n,d,k,ps", [(1000, 37, 10, 300), (777, 128, 1, 10000), (777, 128, 100, 200),
                                      (5, 3, 10, 10000), (1, 1, 1, 10000), (3000, 96, 33, 1000)])
def test_exact_small_ragged(P, torch, pruner, n, d, k, ps):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=n, d=d, nq=13, n_centres=7, seed=n + d))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=ps)
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), k, pruner=pruner)
    torch.cuda.synchronize()
    check_topk(x, q, k, dist, idx, atol=1e-5)


@pytest.mark.parametrize("order,zone", [("dist_to_means", 1), ("dist_to_means", 8), ("dist_to_means", 64),
                                        ("decreasing", 1), ("sequential", 1)])
@pytest.mark.parametrize("first_step,sel,bpi", [(2, 0.2, 0), (1, 0.25, 1), (8, 0.0, 3)])
def test_bond_orders_steps_thresholds(P, torch, order, zone, first_step, sel, bpi):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=5000, d=100, nq=20, n_centres=16, seed=3))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=1500)
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), 10, pruner="bond", order=order, zone_dims=zone,
                                   first_step=first_step, selection_threshold=sel, blocks_per_item=bpi)
    torch.cuda.synchronize()
    check_topk(x, q, 10, dist, idx)


def test_plain_scan_config_10k_d128(P, torch):
    # i.i.d. N(0,1), N=10,000, D=128, 100 queries, k=10, L2 (the plain-scan workload)
    x, q = pdx_synth.make("plain_scan_10k_d128")
    ix = P.pdx_build_layout(_dev(torch, x))
    truth = ok.knn(x, q, 10)
    for pruner in ("none", "bond"):
        dist, idx = P.pdx_search_exact(ix, _dev(torch, q), 10, pruner=pruner)
        torch.cuda.synchronize()
        check_topk(x, q, 10, dist, idx, truth=truth)


def test_host_pointers_match_device(P, torch):
    x, q = pdx_synth.iid_normal(2000, 48, 9, seed=5)
    ix = P.pdx_build_layout(x)                      # host input
    dh, ih = P.pdx_search_exact(ix, q, 7)           # host queries and outputs
    dd, idd = P.pdx_search_exact(ix, _dev(torch, q), 7)
    torch.cuda.synchronize()
    assert isinstance(dh, np.ndarray)
    assert np.array_equal(ih, idd.cpu().numpy())
    assert np.array_equal(dh, dd.cpu().numpy())
    check_topk(x, q, 7, dh, ih)


def test_ties_go_to_lower_index(P, torch):
    rng = np.random.default_rng(7)
    base = rng.standard_normal((50, 16)).astype(np.float32)
    x = np.concatenate([base, base, base])          # every vector three times
    q = base[:6] + 0.01
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=40)
    for pruner in ("none", "bond"):
        dist, idx = P.pdx_search_exact(ix, _dev(torch, q), 3, pruner=pruner)
        got = idx.cpu().numpy()
        for r in range(6):
            assert got[r].tolist() == [r, r + 50, r + 100]


def test_l1_and_inner_product(P, torch):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=3000, d=64, nq=11, n_centres=9, seed=8))
    ix1 = P.pdx_build_layout(_dev(torch, x), metric="l1", partition_size=1000)
    for pruner in ("none", "bond"):
        dist, idx = P.pdx_search_exact(ix1, _dev(torch, q), 10, pruner=pruner)
        torch.cuda.synchronize()
        check_topk(x, q, 10, dist, idx, metric="l1")
    # inner product on arbitrary vectors: linear scan only
    ixp = P.pdx_build_layout(_dev(torch, x), metric="ip", partition_size=1000)
    dist, idx = P.pdx_search_exact(ixp, _dev(torch, q), 10, pruner="none")
    torch.cuda.synchronize()
    check_topk(x, q, 10, dist, idx, metric="ip", atol=1e-4)
    with pytest.raises(P.PdxError) as e:
        P.pdx_search_exact(ixp, _dev(torch, q), 10, pruner="bond")
    assert e.value.status == P.PDX_ERR_UNSUPPORTED
    # unit-norm vectors: pruned IP is searched as L2 (same ranking)
    xu, qu = pdx_synth.embedding_like(4000, 64, 12, n_clusters=32, rank=8)
    ixu = P.pdx_build_layout(_dev(torch, xu), metric="ip", partition_size=1000)
    assert ixu.info.unit_norm == 1
    for pruner in ("none", "bond"):
        dist, idx = P.pdx_search_exact(ixu, _dev(torch, qu), 10, pruner=pruner)
        torch.cuda.synchronize()
        check_topk(xu, qu, 10, dist, idx, metric="ip", atol=2e-6)


def test_empty_and_invalid(P, torch):
    x, q = pdx_synth.iid_normal(100, 8, 3, seed=9)
    ix = P.pdx_build_layout(_dev(torch, x))
    d0, i0 = P.pdx_search_exact(ix, _dev(torch, q[:0]), 5)
    assert tuple(d0.shape) == (0, 5)
    for bad in (0, 1025):
        with pytest.raises(P.PdxError) as e:
            P.pdx_search_exact(ix, _dev(torch, q), bad)
        assert e.value.status == P.PDX_ERR_ARG
    with pytest.raises(P.PdxError):
        P.pdx_search_exact(ix, _dev(torch, q), 5, pruner="ads")      # approximate: IVF only


def test_bond_prunes_and_counts(P, torch):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=20000, d=128, nq=16, n_centres=32, seed=10))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=5000)
    _, _, sn = P.pdx_search_exact(ix, _dev(torch, q), 10, pruner="none", stats=True)
    _, _, sb = P.pdx_search_exact(ix, _dev(torch, q), 10, pruner="bond", stats=True)
    assert sn["values_visited"] == 20000 * 128 * 16
    assert sn["vectors_scanned"] == 20000 * 16 and sn["vectors_pruned"] == 0
    assert sb["values_visited"] < 0.5 * sn["values_visited"]
    assert sb["vectors_scanned"] == 20000 * 16
    assert 0 < sb["vectors_pruned"] < 20000 * 16


def test_bond_threshold_shared_across_partitions(P, torch):
    # 2048 small clusters over 100k vectors: a 10k-vector partition holds only
    # ~5 of a query's ~49 cluster-mates, so no single work item ever sees k
    # near neighbours. The query's threshold must come from everything scanned
    # so far (the paper's one heap per query), or almost nothing gets pruned.
    # The sequential oracle visits 17% of the values with one heap per query
    # and 97.6% with one heap per partition.
    x, q = pdx_synth.embedding_like(100_000, 256, 64, n_clusters=2048, rank=16, seed=91)
    ix = P.pdx_build_layout(_dev(torch, x), metric="ip")
    d, i, sb = P.pdx_search_exact(ix, _dev(torch, q), 10, pruner="bond", stats=True)
    torch.cuda.synchronize()
    check_topk(x, q, 10, d, i, metric="ip")
    assert sb["values_visited"] < 0.4 * 100_000 * 256 * 64, sb


def test_mixture_768_medium(P, torch):
    # the 768-d Gaussian-mixture workload at 100k vectors (oracle on all queries)
    x, q = pdx_synth.make("bond_exact_1m_d768", n=100_000, nq=48)
    ix = P.pdx_build_layout(_dev(torch, x))
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), 10)
    torch.cuda.synchronize()
    check_topk(x, q, 10, dist, idx)


def test_mixture_768_full_size_sampled(P, torch):
    # full size (1M x 768, 1000 queries) in the bench's launch configuration;
    # the oracle checks a sample of the queries one by one
    x, q = pdx_synth.make("bond_exact_1m_d768")
    ix = P.pdx_build_layout(_dev(torch, x))
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), 10)
    torch.cuda.synchronize()
    rows = np.random.default_rng(1).choice(q.shape[0], size=6, replace=False)
    check_topk(x, q, 10, dist, idx, rows=rows)


@pytest.mark.parametrize("scope,zone,d", [("collection", 1, 100), ("collection", 4, 300), ("block", 1, 300),
                                          ("block", 2, 600)])
def test_bond_precomputed_orders(P, torch, scope, zone, d):
    # orders computed once per query (collection means) or per (query, part)
    # (more zones than a warp sorts in-kernel) keep the search exact
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=4000, d=d, nq=12, n_centres=10, seed=d + zone))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=1000)
    for order in ("dist_to_means", "decreasing"):
        dist, idx = P.pdx_search_exact(ix, _dev(torch, q), 10, order=order, zone_dims=zone, means_scope=scope)
        torch.cuda.synchronize()
        check_topk(x, q, 10, dist, idx)


def test_sharded_search_merged_on_device(P, torch):
    # two shards of one collection searched separately, ids made global, lists
    # merged by pdx_merge_topk on the device: the same answer as one index
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=30000, d=96, nq=40, n_centres=16, seed=21))
    half = 13001
    full = P.pdx_build_layout(_dev(torch, x))
    d_full, i_full = P.pdx_search_exact(full, _dev(torch, q), 10)
    parts = []
    for lo, hi in ((0, half), (half, x.shape[0])):
        ix = P.pdx_build_layout(_dev(torch, x[lo:hi]))
        d, i = P.pdx_search_exact(ix, _dev(torch, q), 10)
        parts.append((d, torch.where(i >= 0, i + lo, i)))
    md, mi = P.pdx_merge_topk(torch.stack([p[0] for p in parts]), torch.stack([p[1] for p in parts]))
    torch.cuda.synchronize()
    assert torch.equal(mi, i_full) and torch.equal(md, d_full)
    hd, hi_ = P.pdx_merge_topk(torch.stack([p[0] for p in parts]).cpu().numpy(),
                               torch.stack([p[1] for p in parts]).cpu().numpy())
    assert np.array_equal(hi_, mi.cpu().numpy()) and np.array_equal(hd, md.cpu().numpy())
    check_topk(x, q, 10, md, mi)


@pytest.mark.parametrize("pruner", ["none", "bond"])
def test_k_1024(P, torch, pruner):
    # the largest k the header allows, over several partitions with a ragged tail
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=9000, d=40, nq=6, n_centres=6, seed=27))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=2500)
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), 1024, pruner=pruner)
    torch.cuda.synchronize()
    check_topk(x, q, 1024, dist, idx)


def test_initial_thresholds(P, torch):
    # tau_init at (or above) each query's true k-th distance keeps PDX-BOND
    # exact, with or without tightening (tau_fixed); the fixed run prunes with
    # the true k-th distance from the start, so it visits no more values
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=30000, d=96, nq=32, n_centres=24, seed=28))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=5000)
    td, ti = ok.knn(x, q, 10)
    kth = td[:, -1].astype(np.float32)
    _, _, s0 = P.pdx_search_exact(ix, _dev(torch, q), 10, stats=True)
    for fixed, tau in ((False, kth * np.float32(1.5)), (True, kth), (True, kth * np.float32(1.01))):
        dist, idx, st = P.pdx_search_exact(ix, _dev(torch, q), 10, tau_init=tau, tau_fixed=fixed, stats=True)
        torch.cuda.synchronize()
        check_topk(x, q, 10, dist, idx)
        if fixed:
            assert st["start_values"] == 0
    _, _, sf = P.pdx_search_exact(ix, _dev(torch, q), 10, tau_init=kth, tau_fixed=True, stats=True)
    assert sf["values_visited"] <= s0["values_visited"]
    # a threshold below the k-th distance returns the vectors within it, padded
    low = (td[:, 4] * 1.0001).astype(np.float32)
    dist, idx = P.pdx_search_exact(ix, q, 10, tau_init=low, tau_fixed=True)
    for r in range(q.shape[0]):
        got = [int(v) for v in idx[r] if v >= 0]
        assert got == ti[r, :len(got)].tolist() and len(got) >= 5
    with pytest.raises(P.PdxError):
        P.pdx_search_exact(ix, _dev(torch, q), 10, tau_fixed=True)          # fixed needs tau_init


def test_exact_phase_times(P, torch):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=50000, d=128, nq=200, n_centres=32, seed=29))
    ix = P.pdx_build_layout(_dev(torch, x))
    _, _, st = P.pdx_search_exact(ix, _dev(torch, q), 10, stats=True)
    ph = st["phase_ns"]
    assert ph["start"] > 0 and ph["scan"] > 0 and ph["merge"] > 0
    assert ph["scan"] > ph["merge"]


@pytest.mark.parametrize("clusters", [-1, 40, 300])
def test_start_clusters_keep_bond_exact(P, torch, clusters):
    # START from the query's nearest start clusters (exact distances to their
    # members) gives a real k-th distance, so PDX-BOND stays exact
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=30000, d=64, nq=40, n_centres=30, seed=31))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=3000, start_clusters=clusters)
    for k in (1, 10, 200):
        dist, idx, st = P.pdx_search_exact(ix, _dev(torch, q), k, stats=True)
        torch.cuda.synchronize()
        check_topk(x, q, k, dist, idx)
        assert st["start_values"] > 0


@pytest.mark.parametrize("nq,k,pruner", [(1, 10, "bond"), (3, 100, "bond"), (16, 64, "bond"), (2, 50, "none")])
def test_small_batches_with_long_item_lists(P, torch, nq, k, pruner):
    # a batch of at most 16 queries spreads over many work items, whose lists
    # the final selection filters with many CTAs into a compact buffer; the
    # unpruned scan keeps tau = +inf, so every key passes and the compact buffer
    # overflows into the full-row selection
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=120000, d=32, nq=nq, n_centres=64, seed=61))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=6000)
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), k, pruner=pruner, engine="scan" if pruner == "none" else "auto")
    torch.cuda.synchronize()
    check_topk(x, q, k, dist, idx)
