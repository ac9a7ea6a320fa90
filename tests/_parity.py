"""Comparison of a GPU top-k against the FP64 oracle, with the acceptance
rule of the exact search: the returned id sets equal the oracle's except for
ids whose oracle distance lies within `rtol` (relative) of the oracle's k-th
distance (ties at the boundary), and the returned FP32 distances are within
`rtol` of the FP64 values. Returned ids must be distinct, in range, and carry
their own distance."""
import numpy as np

from oracle import knn as ok

RTOL = 1e-5


def _np(a):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return a.detach().cpu().numpy()
    except ImportError:
        pass
    return np.asarray(a)


def check_topk(x, q, k, gpu_d, gpu_i, metric="l2", rtol=RTOL, atol=0.0, truth=None, rows=None):
    gpu_d = _np(gpu_d).astype(np.float64)
    gpu_i = _np(gpu_i).astype(np.int64)
    x = np.asarray(x, np.float32)
    q = np.asarray(q, np.float32)
    if rows is not None:
        q = q[rows]
        gpu_d, gpu_i = gpu_d[rows], gpu_i[rows]
    od, oi = truth if truth is not None else ok.knn(x, q, k, metric)
    n = x.shape[0]
    valid = min(n, k)
    own = ok.pair_distances(x, q, np.where(gpu_i >= 0, gpu_i, -1), metric)
    for r in range(q.shape[0]):
        g = gpu_i[r]
        assert (g[:valid] >= 0).all() and (g[:valid] < n).all(), f"row {r}: bad ids {g}"
        assert (g[valid:] == -1).all(), f"row {r}: padding {g}"
        assert len(set(g[:valid].tolist())) == valid, f"row {r}: duplicate ids {g}"
        # distances by rank
        np.testing.assert_allclose(gpu_d[r, :valid], od[r, :valid], rtol=rtol, atol=atol,
                                   err_msg=f"row {r} distances by rank")
        # each returned id carries its own distance
        np.testing.assert_allclose(gpu_d[r, :valid], own[r, :valid], rtol=rtol, atol=atol,
                                   err_msg=f"row {r} distance of returned ids")
        if valid < k:
            pad = gpu_d[r, valid:]
            assert np.isinf(pad).all()
        kth = od[r, valid - 1]
        diff = set(g[:valid].tolist()) ^ set(oi[r, :valid].tolist())
        if diff:
            dd = ok.pair_distances(x, q[r:r + 1], np.array([sorted(diff)]), metric)[0]
            tol = rtol * abs(kth) + atol
            assert np.all(np.abs(dd - kth) <= tol), f"row {r}: ids {sorted(diff)} differ beyond the tie tolerance"
