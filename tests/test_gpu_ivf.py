"""GPU parity of the IVF path (Sec. 2.1, Fig. 2; PDXearch over buckets, Sec. 4;
ADSampling and BSA, Sec. 2.3) against the FP64 oracle. The oracle works in the
original space: ADSampling's rotation and BSA's PCA are orthogonal, so
distances, bucket assignments and probe orders are the same there. A
transformed index reports its distances from the original vectors, so they
are held to the same 1e-5 as every other search. The approximate predicates
are compared prune for prune with the sequential PDXearch oracle at fixed
thresholds."""
import math

import numpy as np
import pytest

import pdx_synth
from oracle import knn as ok
from oracle import pdxearch as ops
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
    check_topk(x, q, 10, dist, idx, truth=(truth[0][rows], truth[1][rows]), rows=rows)


def _recall_setup(P, torch, transform):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=40000, d=96, nq=64, n_centres=64, seed=36,
                                                            rotate=True))
    init = np.ascontiguousarray(x[np.random.default_rng(1).choice(40000, size=64, replace=False)])
    # the library draws ADSampling's rotation itself (rotation_seed); k-means is
    # skipped so that the oracle can assign buckets from the same centroids
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=64, kmeans_iters=0, init_centroids=init, transform=transform,
                         rotation_seed=6)
    qd = _dev(torch, q)
    oa, _ = ok.assign(x, init)
    ref_i = ok.knn_probed(x, q, 10, oa, init, 8)[1]     # FP64 oracle over the 8 probed buckets
    _, _, sn = P.pdx_search_ivf(ix, qd, 10, 8, pruner="none", stats=True)
    return x, q, ix, qd, ref_i, sn["values_visited"]


def test_adsampling_keeps_recall(P, torch):
    # eps0 = 2.1 (Sec. 6.1): recall against the oracle's exact search over the
    # same buckets stays high while most values are skipped
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
    assert res[-1][1] >= 0.995            # the exact bound alone (probe near-ties aside)
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
        P.pdx_ivf_build(_dev(torch, x), nlist=501)
    exact = P.pdx_build_layout(_dev(torch, x))
    with pytest.raises(P.PdxError):
        P.pdx_search_ivf(exact, _dev(torch, q), 5, 1)


def test_library_rotation_is_seeded_orthogonal(P, torch):
    # Sec. 2.3: ADSampling's random orthogonal transformation, drawn by the
    # library from rotation_seed when the caller gives none
    x, q, init = _data(n=3000, d=96, nq=16, nlist=12, seed=39)
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=12, kmeans_iters=0, init_centroids=init, transform="ads",
                         rotation_seed=7)
    R = ix.copy_out("rotation").astype(np.float64)
    np.testing.assert_allclose(R.T @ R, np.eye(96), atol=2e-6)
    np.testing.assert_allclose(R @ R.T, np.eye(96), atol=2e-6)
    v = np.random.default_rng(3).standard_normal((5, 96))
    np.testing.assert_allclose(np.linalg.norm(v @ R.T, axis=1), np.linalg.norm(v, axis=1), rtol=2e-6)
    assert abs(np.linalg.det(R)) == pytest.approx(1.0, abs=1e-4)
    # entries of a Haar matrix: mean 0, variance 1/d
    assert abs(R.mean()) < 3.0 / 96 and abs(R.var() * 96 - 1.0) < 0.05
    again = P.pdx_ivf_build(_dev(torch, x), nlist=12, kmeans_iters=0, init_centroids=init, transform="ads",
                            rotation_seed=7).copy_out("rotation")
    other = P.pdx_ivf_build(_dev(torch, x), nlist=12, kmeans_iters=0, init_centroids=init, transform="ads",
                            rotation_seed=8).copy_out("rotation")
    assert np.array_equal(again, R.astype(np.float32))
    assert np.abs(other - R).max() > 0.1
    # the rows keep the original vectors; searches report original-space distances
    np.testing.assert_array_equal(ix.copy_out("rows"), x)
    oa, _ = ok.assign(x, init)
    truth = ok.knn_probed(x, q, 10, oa, init, 4)
    dist, idx = P.pdx_search_ivf(ix, _dev(torch, q), 10, 4, pruner="bond")
    torch.cuda.synchronize()
    rows = _probe_margin_ok(q, init, 4)
    check_topk(x, q, 10, dist, idx, truth=(truth[0][rows], truth[1][rows]), rows=rows)


def _oracle_fixed_tau(xs, qs, k, tau0, pruner, blocks=None, **kw):
    """Per query: (vectors pruned, top-k ids among survivors within tau0) of
    the sequential PDXearch oracle at a fixed threshold. With tau fixed, which
    vectors are pruned depends only on tau and the predicate, not on the order
    of the blocks; storage-order predicates need no blocks at all (one block
    holds every vector), the fused pruner's order and expected distances come
    from each bucket's own vectors."""
    out = []
    allv = blocks if blocks is not None else [np.arange(xs.shape[0])]
    for r in range(qs.shape[0]):
        d, i, st = ops.pdxearch(xs, qs[r], k, allv, pruner=pruner, first_step=4, tau0=float(tau0[r]),
                                tau_fixed=True, **kw)
        keep = [int(v) for v, dd in zip(i, d) if v >= 0 and dd <= tau0[r]]
        out.append((st.vectors_pruned, keep))
    return out


@pytest.mark.parametrize("pruner,knob", [("ads", dict(eps0=2.1)), ("ads", dict(eps0=1.0)),
                                         ("bsa", dict(bsa_m=1.0)), ("bsa", dict(bsa_m=0.5)),
                                         ("ads_bond", dict(eps0=2.1)), ("ads_bond", dict(eps0=1.0))])
def test_approximate_predicates_prune_like_the_oracle(P, torch, pruner, knob):
    # Sec. 2.3 at fixed thresholds: the GPU's ADSampling / BSA tests prune the
    # same vectors as the sequential oracle (which follows the paper's steps).
    # Thresholds within 2e-4 (relative) of a decision may go either way; they
    # are covered by running the oracle at tau0 * (1 -/+ 2e-4).
    n, d, nq, k = 4000, 48, 12, 10
    x, q = pdx_synth.anisotropic_gaussian(n, d, nq, decay=0.93, seed=71)
    x64, q64 = x.astype(np.float64), q.astype(np.float64)
    truth_d, _ = ok.knn(x, q, 3 * k)
    tau0 = truth_d[:, -1].astype(np.float32)          # the 3k-th distance: a real k-th bound
    init = np.ascontiguousarray(x[np.random.default_rng(5).choice(n, size=8, replace=False)])
    if pruner in ("ads", "ads_bond"):
        rot = pdx_synth.random_orthogonal(d, 17)
        ix = P.pdx_ivf_build(_dev(torch, x), nlist=8, kmeans_iters=0, init_centroids=init, transform="ads",
                             rotation=rot, keep_rows=False)
        R = rot.astype(np.float64)
        xs, qs, extra = x64 @ R.T, q64 @ R.T, dict(eps0=knob["eps0"])
        if pruner == "ads_bond":
            # the buckets (nearest initial centroid; rotation does not change it)
            # are the blocks whose means and variances order the dimensions
            oa, _ = ok.assign(x, init)
            extra.update(blocks=[np.flatnonzero(oa == b) for b in range(8)], order="dist_to_means", zone_dims=8)
    else:
        ix = P.pdx_ivf_build(_dev(torch, x), nlist=8, kmeans_iters=0, init_centroids=init, transform="bsa",
                             keep_rows=False)
        mean = x64.mean(axis=0)
        lam, vec = np.linalg.eigh(np.cov(x64.T, bias=True))
        order = np.argsort(-lam, kind="stable")
        lam, vec = np.maximum(lam[order], 0.0), vec[:, order]
        xs, qs = (x64 - mean) @ vec, (q64 - mean) @ vec
        extra = dict(bsa_m=knob["bsa_m"], bsa_lambda=lam)
    lo = _oracle_fixed_tau(xs, qs, k, tau0 * (1 - 2e-4), pruner, **extra)
    mid = _oracle_fixed_tau(xs, qs, k, tau0, pruner, **extra)
    hi = _oracle_fixed_tau(xs, qs, k, tau0 * (1 + 2e-4), pruner, **extra)
    dist, idx, st = P.pdx_search_ivf(ix, _dev(torch, q), k, 8, pruner=pruner, tau_init=_dev(torch, tau0),
                                     tau_fixed=True, stats=True, **knob)
    torch.cuda.synchronize()
    idx = idx.cpu().numpy()
    pruned_hi = sum(p for p, _ in hi)
    pruned_lo = sum(p for p, _ in lo)
    assert pruned_hi <= st["vectors_pruned"] <= pruned_lo, (pruned_hi, st["vectors_pruned"], pruned_lo)
    assert st["vectors_scanned"] == n * nq
    # the predicate prunes a real share at this threshold (not a vacuous test)
    assert sum(p for p, _ in mid) > 0.3 * n * nq
    agree = 0
    for r in range(nq):
        if lo[r][1] != hi[r][1]:
            continue                                      # a decision within the tolerance changes the result
        agree += 1
        got = [int(v) for v in idx[r] if v >= 0]
        assert got == mid[r][1], (r, got, mid[r][1])
    assert agree >= nq // 2


def test_phase_times_cover_the_search(P, torch):
    # pdx_search_stats.phase_ns: the Table 6 breakdown, every phase timed on the stream
    x, q, init = _data(n=20000, d=64, nq=256, nlist=32, seed=43)
    ix = P.pdx_ivf_build(_dev(torch, x), nlist=32, kmeans_iters=2, init_centroids=init, transform="ads")
    _, _, st = P.pdx_search_ivf(ix, _dev(torch, q), 10, 8, pruner="ads", stats=True)
    ph = st["phase_ns"]
    assert set(ph) == {"preprocess", "find_buckets", "start", "scan", "merge"}
    assert all(v > 0 for v in ph.values()), ph
    ex = P.pdx_build_layout(_dev(torch, x))
    _, _, se = P.pdx_search_exact(ex, _dev(torch, q), 10, stats=True)
    assert se["phase_ns"]["find_buckets"] < se["phase_ns"]["scan"]
    assert se["phase_ns"]["start"] > 0 and se["phase_ns"]["scan"] > 0 and se["phase_ns"]["merge"] > 0


def test_ads_bond_recall_and_pruning(P, torch):
    # the fused pruner on a rotated index: recall against the oracle's exact
    # search over the probed buckets stays high, it visits fewer values than
    # plain PDX-BOND, and it is refused on an index without the rotation
    x, q, ix, qd, ref_i, none_vals = _recall_setup(P, torch, "ads")
    _, i, st = P.pdx_search_ivf(ix, qd, 10, 8, pruner="ads_bond", eps0=2.1, stats=True)
    _, _, sb = P.pdx_search_ivf(ix, qd, 10, 8, pruner="bond", stats=True)
    assert ok.recall_at_k(ref_i, i.cpu().numpy()) >= 0.99
    assert st["values_visited"] < sb["values_visited"]
    plain = P.pdx_ivf_build(_dev(torch, x), nlist=16, kmeans_iters=1)
    with pytest.raises(P.PdxError):
        P.pdx_search_ivf(plain, qd, 10, 4, pruner="ads_bond")
