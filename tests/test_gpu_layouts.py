"""Linear scans over the four storage layouts of the layout comparison
(Sec. 3 Fig. 3, the kernel study of Sec. 6.2 / Table 3, N-ary + gather and
DSM in Sec. 7): every layout answers the same exact k-NN, checked against the
FP64 oracle on ragged sizes (partial 64-vector blocks and chunks, odd d)."""
import numpy as np
import pytest

import pdx_synth
from tests._parity import check_topk

pytestmark = pytest.mark.gpu

LAYOUTS = ["pdx", "pdx_kernel", "nary", "nary_gather", "dsm"]


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


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("metric", ["l2", "ip", "l1"])
@pytest.mark.parametrize("n,d,k", [(2500, 36, 10), (1100, 128, 33), (70, 8, 5), (20000, 100, 100)])
def test_layouts_match_oracle(P, torch, layout, metric, n, d, k):
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=n, d=d, nq=9, n_centres=5, seed=n + d + k))
    ix = P.pdx_build_layout(_dev(torch, x), metric=metric, partition_size=1000, keep_dsm=True)
    dist, idx = P.pdx_search_exact(ix, _dev(torch, q), k, pruner="none", engine="scan", layout=layout)
    torch.cuda.synchronize()
    check_topk(x, q, k, dist, idx, metric=metric, atol=1e-5 if metric == "ip" else 0.0)


def test_layout_plain_config_10k_d128(P, torch):
    # the plain-scan workload (10k x 128, 100 queries, k = 10) on every layout
    x, q = pdx_synth.make("plain_scan_10k_d128")
    ix = P.pdx_build_layout(_dev(torch, x), keep_dsm=True)
    ref = None
    for layout in LAYOUTS:
        dist, idx, st = P.pdx_search_exact(ix, _dev(torch, q), 10, pruner="none", engine="scan", layout=layout,
                                           stats=True)
        torch.cuda.synchronize()
        check_topk(x, q, 10, dist, idx)
        assert st["values_visited"] == x.shape[0] * x.shape[1] * q.shape[0]
        if ref is None:
            ref = idx.cpu().numpy()
        assert np.array_equal(idx.cpu().numpy(), ref), layout


def test_layout_requirements(P, torch):
    x, q = pdx_synth.iid_normal(500, 10, 4, seed=3)
    ix = P.pdx_build_layout(_dev(torch, x))
    for layout, why in (("dsm", "keep_dsm"), ("nary", "multiple of 4")):
        with pytest.raises(P.PdxError) as e:
            P.pdx_search_exact(ix, _dev(torch, q), 5, pruner="none", engine="scan", layout=layout)
        assert e.value.status == P.PDX_ERR_UNSUPPORTED and why in str(e.value)
    with pytest.raises(P.PdxError):   # layouts are unpruned scans
        P.pdx_search_exact(ix, _dev(torch, q), 5, pruner="bond", layout="pdx_kernel")
    with pytest.raises(P.PdxError):
        P.pdx_search_exact(ix, _dev(torch, q), 300, pruner="none", layout="pdx_kernel")
