"""GPU parity of the IVF path (Sec. 2.1, Fig. 2; PDXearch over buckets, Sec. 4;
ADSampling and BSA, Sec. 2.3) against the FP64 oracle. The oracle works in the
original space: ADSampling's rotation and BSA's PCA are orthogonal, so
distances, bucket assignments and probe orders are the same there."""
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


def _data(n=6000, d=48, nq=24, nlist=24, seed=31):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=n, d=d, nq=nq, n_centres=nlist, seed=seed))
    init = x[np.random.default_rng(seed).choice(n, size=nlist, replace=False)]
    return x, q, np.ascontiguousarray(init)


def _probe_margin_ok(q, centroids, nprobe, rtol=1e-4):
    """Rows whose nprobe-th and (nprobe+1)-th centroid distances are not near-ties."""
    c = centroids.astype(np.float64)
    ok_rows = []
    for r in range(q.shape[0]):
        dd = np.sort(((c - q[r].astype(np.float64)) ** 2).sum(axis=1))
        if nprobe >= len(dd) or dd[nprobe] - dd[nprobe - 1] > rtol * dd[nprobe]:
            ok_rows.append(r)
    return np.array(ok_rows)


def test_fixed_centroids_assignment_and_buckets(P, torch):
    x, q, init = _data()
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=24, kmeans_iters=0, init_centroids=init)
    a = ix.copy_out("assign")
    oa, od = ok.assign(x, init)
    diff = np.flatnonzero(a != oa)
    if diff.size:       # only FP32 near-ties may differ
        c = init.astype(np.float64)
        for i in diff:
            da = ((x[i] - c[a[i]]) ** 2).sum()
            assert abs(da - od[i]) <= 1e-5 * od[i] + 1e-6
    np.testing.assert_array_equal(ix.copy_out("centroids"), init)
    pb, ids = ix.copy_out("part_blocks"), ix.copy_out("ids")
    for p in range(24):
        members = ids[pb[p] * 64:pb[p + 1] * 64]
        members = members[members >= 0]
        assert (a[members] == p).all()
        assert members.tolist() == sorted(members.tolist())
        assert members.size == (a == p).sum()


def test_kmeans_invariants(P, torch):
    x, q, init = _data(seed=32)
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=24, kmeans_iters=8, init_centroids=init)
    c = ix.copy_out("centroids").astype(np.float64)
    a = ix.copy_out("assign")
    d_all = ((x[:, None, :].astype(np.float64) - c[None]) ** 2).sum(axis=2)
    best = d_all.min(axis=1)
    got = d_all[np.arange(x.shape[0]), a]
    assert np.all(got <= best * (1 + 1e-5) + 1e-6)           # every vector at a nearest centroid
    obj_final = best.sum()
    obj_init = ((x[:, None, :].astype(np.float64) - init[None].astype(np.float64)) ** 2).sum(axis=2).min(axis=1).sum()
    assert obj_final <= obj_init                                # Lloyd never increases the objective


@pytest.mark.parametrize("pruner", ["none", "bond"])
@pytest.mark.parametrize("nprobe", [1, 3, 7])
def test_probed_exact_parity(P, torch, pruner, nprobe):
    x, q, init = _data(seed=33)
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=24, kmeans_iters=0, init_centroids=init)
    oa, _ = ok.assign(x, init)
    truth = ok.knn_probed(x, q, 10, oa, init, nprobe)
    dist, idx = P.pdx_search_ivf(ix, _dev(torch, q), 10, nprobe, pruner=pruner)
    torch.cuda.synchronize()
    rows = _probe_margin_ok(q, init, nprobe)
    check_topk(x, q, 10, dist, idx, truth=(truth[0][rows], truth[1][rows]), rows=rows)


def test_all_buckets_is_brute_force(P, torch):
    x, q, init = _data(seed=34)
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=24, kmeans_iters=3, init_centroids=init)
    dist, idx = P.pdx_search_ivf(ix, _dev(torch, q), 10, 24, pruner="bond")
    torch.cuda.synchronize()
    check_topk(x, q, 10, dist, idx)


@pytest.mark.parametrize("transform,pruner,knob", [("ads", "ads", dict(eps0=1e30)),
                                                   ("bsa", "bsa", dict(bsa_m=1e30)),
                                                   ("ads", "bond", {}), ("bsa", "none", {})])
def test_transformed_indexes_reduce_to_probed_exact(P, torch, transform, pruner, knob):
    # eps0 -> inf never prunes (ADSampling); m -> inf leaves the Cauchy-Schwarz
    # lower bound, which is exact (BSA); BOND/NONE on rotated data are exact
    x, q, init = _data(seed=35)
    rot = pdx_synth.random_orthogonal(x.shape[1], 5) if transform == "ads" else None
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=24, kmeans_iters=0, init_centroids=init, transform=transform,
                         rotation=rot)
    oa, _ = ok.assign(x, init)
    nprobe = 4
    truth = ok.knn_probed(x, q, 10, oa, init, nprobe)
    dist, idx = P.pdx_search_ivf(ix, _dev(torch, q), 10, nprobe, pruner=pruner, **knob)
    torch.cuda.synchronize()
    rows = _probe_margin_ok(q, init, nprobe)
    check_topk(x, q, 10, dist, idx, truth=(truth[0][rows], truth[1][rows]), rows=rows, rtol=2e-5, atol=1e-4)


def _recall_setup(P, torch, transform):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=40000, d=96, nq=64, n_centres=64, seed=36,
                                                            rotate=True))
    init = np.ascontiguousarray(x[np.random.default_rng(1).choice(40000, size=64, replace=False)])
    rot = pdx_synth.random_orthogonal(96, 6) if transform == "ads" else None
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=64, kmeans_iters=4, init_centroids=init, transform=transform,
                         rotation=rot)
    qd = _dev(torch, q)
    ref_d, ref_i = P.pdx_search_ivf(ix, qd, 10, 8, pruner="bond")
    _, _, sn = P.pdx_search_ivf(ix, qd, 10, 8, pruner="none", stats=True)
    return x, q, ix, qd, ref_i.cpu().numpy(), sn["values_visited"]


def test_adsampling_keeps_recall(P, torch):
    # eps0 = 2.1 (Sec. 6.1): recall against the exact search over the same
    # buckets stays high while most values are skipped
    x, q, ix, qd, ref_i, none_vals = _recall_setup(P, torch, "ads")
    _, i, st = P.pdx_search_ivf(ix, qd, 10, 8, pruner="ads", eps0=2.1, stats=True)
    assert ok.recall_at_k(ref_i, i.cpu().numpy()) >= 0.99
    assert st["values_visited"] < 0.5 * none_vals
    truth = ok.knn(x, q, 10)
    assert ok.recall_at_k(truth[1], i.cpu().numpy()) >= 0.8


def test_bsa_multiplier_trades_pruning_for_recall(P, torch):
    # m -> inf leaves only the exact Cauchy-Schwarz test; smaller m prunes more
    # and may lose recall; the paper tunes m to a target recall (Sec. 6.1)
    x, q, ix, qd, ref_i, none_vals = _recall_setup(P, torch, "bsa")
    res = []
    for m in (0.25, 0.5, 1.0, 2.0, 4.0, 1e30):
        _, i, st = P.pdx_search_ivf(ix, qd, 10, 8, pruner="bsa", bsa_m=m, stats=True)
        res.append((m, ok.recall_at_k(ref_i, i.cpu().numpy()), st["values_visited"]))
    assert res[-1][1] == 1.0
    for (m0, r0, v0), (m1, r1, v1) in zip(res, res[1:]):
        assert r1 >= r0 - 0.02, res          # recall grows with m
        assert v1 >= v0 * 0.98, res          # pruning shrinks with m
    # the statistical test adds pruning on top of the exact bound at small m
    assert any(r >= 0.95 and v < res[-1][2] for _, r, v in res), res


def test_pca_projection_properties(P, torch):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=20000, d=40, nq=4, n_centres=16, seed=37))
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=16, kmeans_iters=2, transform="bsa")
    R = ix.copy_out("rotation").astype(np.float64)
    var = ix.copy_out("variances").astype(np.float64)
    np.testing.assert_allclose(R @ R.T, np.eye(40), atol=2e-5)
    assert np.all(np.diff(var) <= 1e-6 * var[0])                      # sorted by decreasing variance
    ref = np.sort(np.linalg.eigvalsh(np.cov(x.astype(np.float64).T, bias=True)))[::-1]
    np.testing.assert_allclose(var, ref, rtol=1e-3, atol=1e-6 * ref[0])


def test_ivf_argument_errors(P, torch):
    x, q, init = _data(n=500, nlist=8, seed=38)
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=8, kmeans_iters=1)
    for bad in (0, 9):
        with pytest.raises(P.PdxError) as e:
            P.pdx_search_ivf(ix, _dev(torch, q), 5, bad)
        assert e.value.status == P.PDX_ERR_ARG
    with pytest.raises(P.PdxError):
        P.pdx_search_ivf(ix, _dev(torch, q), 5, 2, pruner="ads")        # index not rotated
    with pytest.raises(P.PdxError):
        P.pdx_ivf_build(_dev(torch, x), nlist=8, transform="ads")      # rotation missing
    with pytest.raises(P.PdxError):
        P.pdx_ivf_build(_dev(torch, x), nlist=501)
    exact = P.pdx_build_layout(_dev(torch, x))
    with pytest.raises(P.PdxError):
        P.pdx_search_ivf(exact, _dev(torch, q), 5, 1)
