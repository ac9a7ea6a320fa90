"""Pins of the CPU oracle to facts that do not come from the oracle itself:
hand-worked values, inputs built so that the distances are known by
construction, invariants and special cases, and an exact-rational brute force
on tiny inputs. Each test is chosen so that a plausible slip in the oracle (a
dropped dimension, a wrong sign, a transposed operand, a broken tie rule)
fails it."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import knn as ok
from oracle import pdxearch as ops
import pdx_synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_worked_example_distances_and_topk():
    g = _gold("worked_example_4vec.json")
    x = np.array(g["vectors"], np.float32)
    q = np.array([g["query"]], np.float32)
    d, i = ok.knn(x, q, 4, "l2")
    assert i[0].tolist() == [0, 1, 2, 3]
    assert d[0].tolist() == sorted(g["l2"])
    assert ok.knn(x, q, 2)[1][0].tolist() == g["top2_ids"]
    assert ok.knn(x, q, 3)[1][0].tolist() == g["top3_ids"]
    di, ii = ok.knn(x, q, 2, "ip")
    assert ii[0].tolist() == g["top2_ip_ids"] and di[0].tolist() == [3.0, 1.0]
    dl1, il1 = ok.knn(x, q, 4, "l1")
    assert sorted(dl1[0].tolist()) == sorted(g["l1"])


def test_worked_example_bond_prune_events():
    g = _gold("worked_example_4vec.json")["bond"]
    w = _gold("worked_example_4vec.json")
    x = np.array(w["vectors"], np.float64)
    q = np.array(w["query"], np.float64)
    d, i, st = ops.pdxearch(x, q, g["k"], [np.array(b) for b in g["blocks"]], pruner="bond",
                            order=g["order"], first_step=g["first_step"])
    assert i.tolist() == w["top2_ids"]
    assert [list(e) for e in st.prune_events] == g["prune_events"]


def test_constructed_distances_l2():
    # integer query, vectors q + r_i * e_{j_i}: distance is exactly r_i^2, the
    # ranking is known by construction (not computed by any formula here)
    rng = np.random.default_rng(1)
    d = 7
    q = rng.integers(-5, 6, size=d).astype(np.float32)
    radii = [3, -1, 4, 2, -6, 5, 0.5, -2.5]
    dims = [6, 0, 3, 6, 1, 2, 5, 4]          # includes the last dimension (index d-1)
    x = np.stack([q + r * np.eye(d, dtype=np.float32)[j] for r, j in zip(radii, dims)])
    dist, idx = ok.knn(x, q[None], len(radii))
    expect = [6, 1, 3, 7, 0, 2, 5, 4]         # |r| = 0.5, 1, 2, 2.5, 3, 4, 5, 6
    assert idx[0].tolist() == expect
    assert dist[0].tolist() == [0.25, 1, 4, 6.25, 9, 16, 25, 36]


def test_last_dimension_counts():
    # vectors identical to the query except in the final dimension
    q = np.zeros((1, 5), np.float32)
    x = np.zeros((3, 5), np.float32)
    x[0, 4] = 3.0
    x[1, 4] = -1.0
    x[2, 0] = 2.0
    dist, idx = ok.knn(x, q, 3)
    assert idx[0].tolist() == [1, 2, 0]
    assert dist[0].tolist() == [1.0, 4.0, 9.0]


def test_sign_of_difference():
    # (v - q)^2, not (v + q)^2: the mirrored vector -q is the farthest one
    q = np.array([[1.0, -2.0, 3.0]], np.float32)
    x = np.array([[-1.0, 2.0, -3.0], [1.0, -2.0, 3.0], [0.0, 0.0, 0.0]], np.float32)
    dist, idx = ok.knn(x, q, 3)
    assert idx[0].tolist() == [1, 2, 0]
    assert dist[0].tolist() == [0.0, 14.0, 56.0]


def test_query_not_transposed_nonsquare():
    # n != d != nq: query j's nearest neighbour is the vector planted at it
    rng = np.random.default_rng(2)
    nq, n, d = 3, 11, 5
    q = rng.integers(-3, 4, size=(nq, d)).astype(np.float32)
    x = rng.integers(20, 30, size=(n, d)).astype(np.float32)
    plant = [7, 2, 10]
    for j, p in enumerate(plant):
        x[p] = q[j]
    dist, idx = ok.knn(x, q, 1)
    assert idx[:, 0].tolist() == plant
    assert dist[:, 0].tolist() == [0.0, 0.0, 0.0]


def test_inner_product_closed_form():
    d = 6
    q = np.zeros((1, d), np.float32)
    q[0, 2] = 1.0
    scales = [0.5, -3.0, 2.0, 7.0, 2.0]
    x = np.stack([s * np.eye(d, dtype=np.float32)[2] for s in scales])
    dist, idx = ok.knn(x, q, 5, "ip")
    assert idx[0].tolist() == [3, 2, 4, 0, 1]      # 7, 2 (id 2), 2 (id 4), 0.5, -3
    assert dist[0].tolist() == [7.0, 2.0, 2.0, 0.5, -3.0]


def test_ties_break_to_lower_index():
    v = np.array([1.0, 2.0, 3.0], np.float32)
    x = np.stack([v + 1, v, v + 1, v, v - 1])
    dist, idx = ok.knn(x, v[None], 5)
    assert idx[0].tolist() == [1, 3, 0, 2, 4]


def test_padding_when_n_below_k():
    x = np.zeros((2, 3), np.float32)
    q = np.ones((1, 3), np.float32)
    dist, idx = ok.knn(x, q, 4)
    assert idx[0].tolist() == [0, 1, -1, -1]
    assert math.isinf(dist[0, 2]) and dist[0, 2] > 0
    di, ii = ok.knn(x, q, 4, "ip")
    assert math.isinf(di[0, 3]) and di[0, 3] < 0


def _rational_topk(x, q, k):
    res = []
    for qq in q:
        ds = []
        for i, v in enumerate(x):
            s = sum((Fraction(float(a)) - Fraction(float(b))) ** 2 for a, b in zip(v, qq))
            ds.append((s, i))
        ds.sort()
        res.append([i for _, i in ds[:k]])
    return res


def test_exhaustive_rational_bruteforce_tiny():
    # every query/vector set of a tiny grid-valued problem, in exact rationals
    rng = np.random.default_rng(3)
    for trial in range(30):
        n, d, nq = int(rng.integers(1, 12)), int(rng.integers(1, 5)), 3
        x = (rng.integers(-4, 5, size=(n, d)) / 2).astype(np.float32)
        q = (rng.integers(-4, 5, size=(nq, d)) / 2).astype(np.float32)
        k = int(rng.integers(1, n + 1))
        _, idx = ok.knn(x, q, k)
        assert idx.tolist() == _rational_topk(x, q, k)


def test_probed_oracle_restricts_to_nearest_buckets():
    # two far-apart buckets; nprobe=1 must only return members of the nearer one
    c = np.array([[0, 0], [100, 100]], np.float32)
    x = np.array([[1, 0], [0, 2], [99, 100], [100, 98], [50, 50]], np.float32)
    a = np.array([0, 0, 1, 1, 1], np.int32)      # id 4 deliberately in bucket 1
    q = np.array([[10, 10]], np.float32)
    _, idx1 = ok.knn_probed(x, q, 3, a, c, 1)
    assert idx1[0].tolist() == [1, 0, -1]       # 164 < 181
    _, idx2 = ok.knn_probed(x, q, 3, a, c, 2)
    _, full = ok.knn(x, q, 3)
    assert idx2.tolist() == full.tolist()


def test_assign_by_construction():
    rng = np.random.default_rng(4)
    c = (rng.standard_normal((6, 9)) * 50).astype(np.float32)
    lab = rng.integers(0, 6, size=200)
    x = (c[lab] + rng.standard_normal((200, 9)).astype(np.float32)).astype(np.float32)
    a, _ = ok.assign(x, c)
    assert (a == lab).all()
    # a point equidistant from centroids 1 and 4 goes to the lower id
    mid = ((c[1] + c[4]) / 2)[None]
    c2 = c.copy()
    a2, _ = ok.assign(np.zeros((1, 9), np.float32), np.stack([c2[0] * 0 + 1, c2[0] * 0 - 1]))
    assert a2[0] == 0
    del mid


def test_kmeans_objective_nonincreasing_and_recovers_means():
    rng = np.random.default_rng(5)
    true = (rng.standard_normal((4, 3)) * 20).astype(np.float32)
    lab = np.repeat(np.arange(4), 50)
    x = (true[lab] + rng.standard_normal((200, 3))).astype(np.float32)
    init = x[[0, 50, 100, 150]]
    c, a, obj = ok.kmeans(x, init, 10)
    assert np.all(np.diff(obj) <= 1e-9 * obj[0])
    assert (a == lab).all()
    for j in range(4):
        np.testing.assert_allclose(c[j], x[lab == j].astype(np.float64).mean(axis=0), rtol=0, atol=1e-9)


def test_recall_definition():
    t = np.array([[1, 2, 3, 4]])
    assert ok.recall_at_k(t, np.array([[4, 3, 9, -1]])) == 0.5
    assert ok.recall_at_k(t, t) == 1.0


@pytest.mark.parametrize("order,zone", [("dist_to_means", 1), ("dist_to_means", 4), ("decreasing", 1),
                                        ("sequential", 1)])
@pytest.mark.parametrize("first_step,sel", [(2, 0.2), (1, 0.5), (4, 0.05)])
def test_pdxearch_bond_is_exact(order, zone, first_step, sel):
    # PDX-BOND prunes only with the partial distance, a lower bound, so for any
    # visit order, step schedule and selection threshold the result must be the
    # brute-force top-k (Sec. 5: "exact").
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=700, d=24, nq=5, n_centres=8, seed=11))
    k = 7
    blocks = ops.partitions(700, 64)
    _, truth = ok.knn(x, q, k)
    for j in range(q.shape[0]):
        _, idx, st = ops.pdxearch(x, q[j], k, blocks, pruner="bond", order=order, zone_dims=zone,
                                  first_step=first_step, selection_threshold=sel)
        assert idx.tolist() == truth[j].tolist()
        assert st.values_visited <= 700 * 24


def test_pdxearch_bond_prunes_on_clustered_data():
    # 16 clusters of ~125 vectors: the 10 nearest neighbours share the query's
    # cluster, so vectors of other clusters exceed tau after a few dimensions
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=2000, d=64, nq=3, n_centres=16, seed=12))
    blocks = ops.partitions(2000, 256)
    for j in range(3):
        _, _, st = ops.pdxearch(x, q[j], 10, blocks)
        assert st.values_visited < 0.5 * 2000 * 64      # pruning power > 50%


def test_pdxearch_ads_bsa_special_cases_reduce_to_exact():
    # eps0 -> infinity never prunes (ADSampling); m -> infinity leaves only the
    # Cauchy-Schwarz lower bound, which is exact (BSA reading)
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=500, d=32, nq=3, n_centres=6, seed=13))
    rot = pdx_synth.random_orthogonal(32, 99)
    xr, qr = x @ rot.T, q @ rot.T
    blocks = ops.partitions(500, 64)
    _, truth = ok.knn(xr, qr, 5)
    lam = np.var(xr.astype(np.float64), axis=0)
    for j in range(3):
        _, i1, _ = ops.pdxearch(xr, qr[j], 5, blocks, pruner="ads", eps0=1e30)
        assert i1.tolist() == truth[j].tolist()
        _, i2, _ = ops.pdxearch(xr, qr[j], 5, blocks, pruner="bsa", bsa_m=1e30, bsa_lambda=lam)
        assert i2.tolist() == truth[j].tolist()


def test_ads_at_finite_eps_keeps_high_recall():
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=3000, d=64, nq=8, seed=14, rotate=True))
    rot = pdx_synth.random_orthogonal(64, 5)
    xr, qr = x @ rot.T, q @ rot.T
    blocks = ops.partitions(3000, 256)
    _, truth = ok.knn(xr, qr, 10)
    found = [ops.pdxearch(xr, qr[j], 10, blocks, pruner="ads", eps0=2.1)[1] for j in range(8)]
    assert ok.recall_at_k(truth, np.stack(found)) >= 0.95


def test_visit_order_rules():
    q = np.array([0.0, 5.0, -1.0, 5.0])
    mu = np.array([0.0, 0.0, 3.0, 0.0])
    # (q-mu)^2 = 0, 25, 16, 25 -> dims 1, 3 (tie -> lower first), 2, 0
    assert ops.visit_order(q, mu, "dist_to_means").tolist() == [1, 3, 2, 0]
    # decreasing query value: 5 (dim 1), 5 (dim 3), 0, -1
    assert ops.visit_order(q, mu, "decreasing").tolist() == [1, 3, 0, 2]
    # zones of 2: zone 0 = {0,1} score 25, zone 1 = {2,3} score 41 -> zone 1 first
    assert ops.visit_order(q, mu, "dist_to_means", 2).tolist() == [2, 3, 0, 1]
    assert ops.step_schedule(10, 2) == [2, 4, 4]
    assert ops.step_schedule(768, 2) == [2, 4, 8, 16, 32, 64, 128, 256, 258]


def test_random_orthogonal_is_orthogonal():
    p = pdx_synth.random_orthogonal(48, 3).astype(np.float64)
    np.testing.assert_allclose(p.T @ p, np.eye(48), atol=1e-6)
    v = np.random.default_rng(0).standard_normal(48)
    assert abs(np.linalg.norm(p @ v) - np.linalg.norm(v)) < 1e-6 * np.linalg.norm(v)


def _worked(name):
    return _gold("ads_bsa_worked.json")[name]


def test_ads_predicate_hand_worked_events():
    # tests/golden/ads_bsa_worked.json "ads": every prune event worked out by
    # hand from Sec. 2.3's hypothesis test at a fixed tau. A predicate that
    # never fires, an inverted D/d, a dropped square or eps0/d instead of
    # eps0/sqrt(d) each moves or removes one of the two events.
    g = _worked("ads")
    x = np.array(g["vectors"], np.float64)
    q = np.array(g["query"], np.float64)
    d, i, st = ops.pdxearch(x, q, g["k"], [np.arange(x.shape[0])], pruner="ads", eps0=g["eps0"],
                            first_step=g["first_step"], tau0=g["tau0"])
    assert [list(e) for e in st.prune_events] == g["prune_events"]
    assert i.tolist() == g["top_ids"]
    assert d.tolist() == g["top_dists"]
    # a larger eps0 widens the test: x2 is no longer pruned at d=6
    _, _, st2 = ops.pdxearch(x, q, g["k"], [np.arange(x.shape[0])], pruner="ads", eps0=4.0,
                             first_step=g["first_step"], tau0=g["tau0"])
    assert [e[1] for e in st2.prune_events] == []


def test_bsa_predicate_hand_worked_events():
    # "bsa": one vector pruned only by the error-quantile test (x0), one only
    # by the Cauchy-Schwarz bound at each check point (x3 at d=2, x5 at d=6),
    # and one (x4) that survives only if ||q_r|| enters with the right sign.
    # F(d) differs from d/D here, so a fraction of dimensions in place of the
    # fraction of variance moves x0's event.
    g = _worked("bsa")
    x = np.array(g["vectors"], np.float64)
    q = np.array(g["query"], np.float64)
    d, i, st = ops.pdxearch(x, q, g["k"], [np.arange(x.shape[0])], pruner="bsa", bsa_m=g["m"],
                            bsa_lambda=np.array(g["variances"], np.float64), first_step=g["first_step"],
                            tau0=g["tau0"])
    assert [list(e) for e in st.prune_events] == g["prune_events"]
    assert i.tolist() == g["top_ids"]
    assert d.tolist() == g["top_dists"]


def test_ads_bond_predicate_hand_worked_events():
    # "ads_bond": the fused predicate (PDX-BOND order + mass-calibrated
    # hypothesis test + PDX-BOND's exact test). At tau = 4.01 x0 is pruned by
    # the test alone at d=1; at tau = 4.2 it survives d=1 and BOND prunes it
    # at d=3. Dropping the variance term from E_j, the square of the factor,
    # or the query-aware order each changes one of the two event lists.
    g = _worked("ads_bond")
    x = np.array(g["vectors"], np.float64)
    q = np.array(g["query"], np.float64)
    for case in g["cases"]:
        d, i, st = ops.pdxearch(x, q, g["k"], [np.arange(x.shape[0])], pruner="ads_bond", eps0=g["eps0"],
                                first_step=g["first_step"], tau0=case["tau0"])
        assert [list(e) for e in st.prune_events] == case["prune_events"]
        assert i.tolist() == g["top_ids"] and d.tolist() == g["top_dists"]


def test_ads_bond_reduces_to_adsampling_without_reordering():
    # equal expected contributions and storage order: F_q(d) = d / D, so the
    # fused statistical test is ADSampling's; the fused predicate prunes every
    # vector ADSampling prunes, and any other vector it prunes is one whose
    # distance exceeds tau (PDX-BOND's exact test)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((300, 16))
    q = np.zeros(16)
    x -= x.mean(axis=0)
    x /= x.std(axis=0)                      # mean 0, variance 1 in every dimension
    blocks = [np.arange(300)]
    for tau in (8.0, 14.0):
        _, _, a = ops.pdxearch(x, q, 5, blocks, pruner="ads_bond", order="sequential", eps0=1.5, first_step=2,
                               tau0=tau)
        _, _, b = ops.pdxearch(x, q, 5, blocks, pruner="ads", eps0=1.5, first_step=2, tau0=tau)
        bond_only = {(e[1]) for e in a.prune_events} - {(e[1]) for e in b.prune_events}
        # every extra prune of the fused test is one PDX-BOND's exact test makes
        for v in bond_only:
            assert ((x[v] - q) ** 2).sum() > tau
        assert {e[1] for e in b.prune_events} <= {e[1] for e in a.prune_events}


def test_cs_ip_predicate_hand_worked_events():
    # tests/golden/cs_ip_worked.json: the exact Cauchy-Schwarz bound for the
    # inner product at a fixed tau. A flipped sign loses the result; ||q|| or
    # ||x|| in place of the unvisited norms keeps x6 at d=3; an unvisited set
    # that starts one dimension late prunes x7 at d=1.
    g = _gold("cs_ip_worked.json")
    x = np.array(g["vectors"], np.float64)
    q = np.array(g["query"], np.float64)
    d, i, st = ops.pdxearch(x, q, g["k"], [np.arange(x.shape[0])], pruner="cs_ip", metric="ip",
                            first_step=g["first_step"], tau0=g["tau0"], tau_fixed=True)
    assert [list(e) for e in st.prune_events] == g["prune_events"]
    assert i.tolist() == g["top_ids"]
    assert d.tolist() == g["top_dists"]


@pytest.mark.parametrize("first_step,sel", [(1, 0.2), (4, 0.2), (2, 0.6)])
def test_cs_ip_is_exact_for_any_norms(first_step, sel):
    # the bound holds for every vector, so the pruned search returns the brute
    # force inner-product top-k, with norms spread over two orders of magnitude
    rng = np.random.default_rng(31)
    n, d, k = 900, 20, 9
    x = rng.standard_normal((n, d)) * (0.5 ** np.arange(d) * 3.0) * np.exp(rng.uniform(-2.3, 2.3, (n, 1)))
    q = rng.standard_normal((4, d)) * (0.5 ** np.arange(d) * 3.0)
    blocks = ops.partitions(n, 128)
    tdist, truth = ok.knn(x.astype(np.float32), q.astype(np.float32), k, metric="ip")
    for j in range(q.shape[0]):
        dd, idx, st = ops.pdxearch(x.astype(np.float32), q[j].astype(np.float32), k, blocks, pruner="cs_ip",
                                   metric="ip", first_step=first_step, selection_threshold=sel)
        assert idx.tolist() == truth[j].tolist()
        np.testing.assert_allclose(-dd, tdist[j], rtol=1e-12)
        # energy decays with the dimension: most vectors end early
        assert st.values_visited < 0.6 * n * d


def test_cs_ip_with_a_query_zero_beyond_the_check_is_the_exact_test():
    # ||q_r|| = 0 after the first check point: the bound equals -q.x, so a
    # vector is pruned there exactly when its -q.x exceeds tau
    rng = np.random.default_rng(32)
    x = rng.standard_normal((200, 8))
    q = np.array([1.5, -2.0, 0, 0, 0, 0, 0, 0])
    tau = -1.0
    _, _, st = ops.pdxearch(x, q, 3, [np.arange(200)], pruner="cs_ip", metric="ip", first_step=2, tau0=tau,
                            tau_fixed=True)
    pruned_at_2 = {e[1] for e in st.prune_events if e[2] == 2}
    assert pruned_at_2 == {v for v in range(200) if -(x[v] @ q) > tau}
