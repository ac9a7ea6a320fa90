"""The exact-mode invariant checked on the GPU itself: the scan records every
vector it carries through all D dimensions (`finished_log`), and every query's
true top-k (the FP64 oracle's) must be among them, i.e. no prune test of the
PDXearch scan discarded a true neighbour. Complements the result parity tests,
which see only the final top-k."""
import numpy as np
import pytest

import pdx_synth
from oracle import knn as ok

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


def _logged(torch, P, ix, x, q, k, cap, **kw):
    log = torch.zeros(cap, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    o = P.search_opts(finished_log=log, finished_count=cnt, **kw)
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), k, opts=o)
    torch.cuda.synchronize()
    n_log = int(cnt.item())
    assert n_log <= cap, "finished_log overflowed: raise the test's capacity"
    entries = log[:n_log].cpu().numpy().astype(np.uint64)
    per_query = [set() for _ in range(q.shape[0])]
    qs, ids = (entries >> np.uint64(32)).astype(np.int64), (entries & np.uint64(0xffffffff)).astype(np.int64)
    for a, b in zip(qs, ids):
        assert 0 <= a < q.shape[0] and 0 <= b < x.shape[0]
        assert b not in per_query[a], "a vector finished twice for one query"
        per_query[a].add(int(b))
    return per_query, dist.cpu().numpy(), idx.cpu().numpy(), n_log


def _check_invariant(x, q, k, per_query, idx, metric="l2", rtol=1e-5):
    td, ti = ok.knn(x, q, k, metric)
    for r in range(q.shape[0]):
        missing = set(ti[r].tolist()) - per_query[r]
        if missing:
            # only a tie at the k-th distance may be replaced by an equal vector
            dd = ok.pair_distances(x, q[r:r + 1], np.array([sorted(missing)]), metric)[0]
            assert np.all(np.abs(dd - td[r, -1]) <= rtol * abs(td[r, -1])), (r, sorted(missing))
        # every returned vector was carried through all dimensions
        assert set(int(v) for v in idx[r] if v >= 0) <= per_query[r], r


@pytest.mark.parametrize("keep_rows", [True, False])
def test_no_true_neighbour_is_pruned_bond(P, torch, keep_rows):
    n, d, nq, k = 30000, 64, 24, 10
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=n, d=d, nq=nq, n_centres=24, seed=71))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=4000, keep_rows=keep_rows)
    per_query, _, idx, n_log = _logged(torch, P, ix, x, q, k, cap=nq * n, pruner="bond")
    _check_invariant(x, q, k, per_query, idx)
    # the scan prunes: far fewer vectors finish than the collection holds
    assert n_log < 0.2 * n * nq


def test_no_true_neighbour_is_pruned_at_k_100_with_start_clusters(P, torch):
    n, d, nq, k = 80000, 48, 8, 100
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=n, d=d, nq=nq, n_centres=40, seed=72))
    ix = P.pdx_build_layout(_dev(torch, x), partition_size=5000)      # n >= 65536: START from start clusters
    per_query, _, idx, _ = _logged(torch, P, ix, x, q, k, cap=nq * n, pruner="bond")
    _check_invariant(x, q, k, per_query, idx)


def test_no_true_neighbour_is_pruned_cs_ip(P, torch):
    n, d, nq, k = 20000, 48, 16, 10
    x, q = pdx_synth.mips_vectors(n, d, nq, decay=0.9, norm_spread=1.0, seed=73)
    ix = P.pdx_build_layout(_dev(torch, x), metric="ip", partition_size=3000, cs_first_step=4)
    per_query, _, idx, n_log = _logged(torch, P, ix, x, q, k, cap=nq * n, pruner="cs_ip")
    _check_invariant(x, q, k, per_query, idx, metric="ip")
    assert n_log < 0.5 * n * nq


def test_finished_log_arguments(P, torch):
    x, q = pdx_synth.iid_normal(2000, 16, 4)
    xd, qd = _dev(torch, x), _dev(torch, q)
    log = torch.zeros(100, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    lp = P.pdx_build_layout(xd, storage="fp8")
    with pytest.raises(P.PdxError):
        P.pdx_search_exact(lp, qd, 5, opts=P.search_opts(finished_log=log, finished_count=cnt))
    f32 = P.pdx_build_layout(xd)
    with pytest.raises(P.PdxError):
        P.pdx_search_exact(f32, qd, 5, opts=P.search_opts(pruner="none", finished_log=log, finished_count=cnt))
    # a small capacity: entries beyond it are counted, not stored
    P.pdx_search_exact(f32, qd, 5, opts=P.search_opts(finished_log=log[:3], finished_count=cnt))
    torch.cuda.synchronize()
    assert int(cnt.item()) >= 4 * 5
    assert (log[3:].cpu().numpy() == 0).all()
