"""GPU parity of the exact inner-product pruner with the Cauchy-Schwarz bound
(PDX_PRUNE_CS_IP) against the FP64 oracle, through the C ABI: exact results
for vectors of any norm, prune-for-prune agreement with the oracle at fixed
thresholds, and the argument checks."""
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


def _ip_atol(x, q):
    # An FP32 inner product is within d * 2^-24 * sum_j |q_j x_j| <= d * 2^-24
    # ||q|| ||x|| of the exact one, however small q.x is (cancellation), so a
    # result near zero is held to that absolute bound besides the relative one.
    d = x.shape[1]
    return d * 2.0 ** -24 * float(np.linalg.norm(q, axis=1).max()) * float(np.linalg.norm(x, axis=1).max())


@pytest.mark.parametrize("n,d,k,ps,fs", [(20000, 48, 10, 3000, 4), (7777, 64, 100, 10000, 2),
                                         (3001, 40, 1, 512, 8), (50, 12, 64, 10000, 4)])
def test_cs_ip_is_exact(P, torch, n, d, k, ps, fs):
    # several partitions with a ragged tail, k from 1 to above n; norms spread
    # over e^[-1, 1]
    x, q = pdx_synth.mips_vectors(n, d, 64, decay=0.9, norm_spread=1.0, seed=81 + d)
    ix = P.pdx_build_layout(_dev(torch, x), metric="ip", partition_size=ps, cs_first_step=fs)
    dist, idx, st = P.pdx_search_exact(ix, _dev(torch, q), k, pruner="cs_ip", stats=True)
    torch.cuda.synchronize()
    check_topk(x, q, k, dist, idx, metric="ip", atol=_ip_atol(x, q))
    assert st["vectors_scanned"] == n * 64


def test_cs_ip_prunes_when_the_energy_is_in_the_leading_dimensions(P, torch):
    n, d, nq = 60000, 96, 256
    x, q = pdx_synth.mips_vectors(n, d, nq, decay=0.93, norm_spread=1.0, seed=90)
    ix = P.pdx_build_layout(_dev(torch, x), metric="ip", cs_first_step=4)
    qd = _dev(torch, q)
    dc, ic, sc = P.pdx_search_exact(ix, qd, 10, pruner="cs_ip", stats=True)
    dn, inn, sn = P.pdx_search_exact(ix, qd, 10, pruner="none", stats=True)
    torch.cuda.synchronize()
    check_topk(x, q, 10, dc, ic, metric="ip", atol=_ip_atol(x, q))
    assert np.array_equal(ic.cpu().numpy(), inn.cpu().numpy())
    # the bound ends most vectors well before the last dimension
    assert sc["values_visited"] < 0.5 * sn["values_visited"], (sc["values_visited"], sn["values_visited"])


def _oracle_fixed_tau(x, q, k, taus, blocks, first_step):
    out = []
    for r in range(q.shape[0]):
        d, i, st = ops.pdxearch(x, q[r], k, blocks, pruner="cs_ip", metric="ip", first_step=first_step,
                                tau0=float(taus[r]), tau_fixed=True)
        keep = [int(v) for v, dd in zip(i, d) if v >= 0 and dd <= taus[r]]
        out.append((st.vectors_pruned, keep))
    return out


def test_cs_ip_prunes_like_the_oracle(P, torch):
    # at a fixed threshold per query (the 3k-th best -q.x, a real bound) the
    # GPU prunes the vectors the FP64 oracle prunes. Decisions within the GPU's
    # rounding margin (D * 2^-23 of ||q_r|| ||x_r|| + ||q|| ||x||, far below
    # 1e-3 of tau here) may go either way, so the oracle runs at tau -/+ 1e-3 |tau|.
    n, d, nq, k, ps, fs = 6000, 48, 12, 10, 2000, 4
    x, q = pdx_synth.mips_vectors(n, d, nq, decay=0.9, norm_spread=0.7, seed=95)
    x64, q64 = x.astype(np.float64), q.astype(np.float64)
    tdist, _ = ok.knn(x, q, 3 * k, metric="ip")
    tau0 = (-tdist[:, -1]).astype(np.float32)            # -q.x of the 3k-th best vector
    blocks = ops.partitions(n, ps)
    lo = _oracle_fixed_tau(x64, q64, k, tau0 - 1e-3 * np.abs(tau0), blocks, fs)   # prunes more
    mid = _oracle_fixed_tau(x64, q64, k, tau0, blocks, fs)
    hi = _oracle_fixed_tau(x64, q64, k, tau0 + 1e-3 * np.abs(tau0), blocks, fs)   # prunes less
    # no rows: every survivor is tested at every check point, as in the oracle
    ix = P.pdx_build_layout(_dev(torch, x), metric="ip", partition_size=ps, cs_first_step=fs, keep_rows=False)
    dist, idx, st = P.pdx_search_exact(ix, _dev(torch, q), k, pruner="cs_ip", tau_init=_dev(torch, tau0),
                                       tau_fixed=True, stats=True)
    torch.cuda.synchronize()
    pruned_hi = sum(p for p, _ in hi)
    pruned_lo = sum(p for p, _ in lo)
    assert pruned_hi <= st["vectors_pruned"] <= pruned_lo, (pruned_hi, st["vectors_pruned"], pruned_lo)
    assert sum(p for p, _ in mid) > 0.3 * n * nq          # the bound prunes a real share
    idx = idx.cpu().numpy()
    agree = 0
    for r in range(nq):
        if lo[r][1] != hi[r][1]:
            continue
        agree += 1
        got = [int(v) for v in idx[r] if v >= 0]
        assert got == mid[r][1], (r, got, mid[r][1])
    assert agree >= nq // 2


def test_cs_ip_schedule_is_the_index_one(P, torch):
    # the stored norms fix the check points: a search asking for another first
    # step runs the index's schedule and stays exact
    x, q = pdx_synth.mips_vectors(5000, 40, 16, seed=97)
    ix = P.pdx_build_layout(_dev(torch, x), metric="ip", cs_first_step=2)
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), 10, pruner="cs_ip", first_step=8)
    torch.cuda.synchronize()
    check_topk(x, q, 10, dist, idx, metric="ip", atol=_ip_atol(x, q))


def test_cs_ip_through_the_server(P, torch):
    x, q = pdx_synth.mips_vectors(12000, 32, 40, seed=98)
    ix = P.pdx_build_layout(_dev(torch, x), metric="ip", cs_first_step=4)
    srv = P.Server([ix], k=7, max_batch=64, use_graphs=True, autotune=True, pruner="cs_ip")
    try:
        for b in (1, 5, 40):
            dist, idx = srv.search(0, _dev(torch, q[:b]))
            torch.cuda.synchronize()
            check_topk(x, q[:b], 7, dist, idx, metric="ip", atol=_ip_atol(x, q))
    finally:
        srv.free()


def test_cs_ip_argument_errors(P, torch):
    x, q = pdx_synth.mips_vectors(600, 16, 4, seed=99)
    xd, qd = _dev(torch, x), _dev(torch, q)
    l2 = P.pdx_build_layout(xd)
    with pytest.raises(P.PdxError):
        P.pdx_search_exact(l2, qd, 5, pruner="cs_ip")              # an L2 index
    ip = P.pdx_build_layout(xd, metric="ip")
    with pytest.raises(P.PdxError):
        P.pdx_search_exact(ip, qd, 5, pruner="cs_ip")              # no stored norms
    with pytest.raises(P.PdxError):
        P.pdx_search_exact(ip, qd, 5, pruner="bond")               # partial inner products do not bound
    with pytest.raises(P.PdxError):
        P.pdx_build_layout(xd, cs_first_step=4)                    # norms on an L2 index
    with pytest.raises(P.PdxError):
        P.pdx_build_layout(xd, metric="ip", storage="bf16", cs_first_step=4)
    with pytest.raises(P.PdxError):
        P.pdx_build_layout(xd, metric="ip", cs_first_step=17)      # beyond d
