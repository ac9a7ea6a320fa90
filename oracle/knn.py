"""ctypes wrapper over the C brute-force oracle (``knn_oracle.c``).

Test infrastructure only (see the package docstring). ``build()`` compiles the
C file with gcc into ``oracle/_build/liboracle.so``; it has no CUDA in it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

METRICS = {"l2": 0, "ip": 1, "l1": 2}


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, pthreads). Idempotent."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.oracle_knn.argtypes = [p, i64, i32, p, i64, i32, i32, i32, p, p]
            lib.oracle_knn_probed.argtypes = [p, i64, i32, p, i64, i32, i32, p, p, i32, i32, i32, p, p]
            lib.oracle_assign.argtypes = [p, i64, i32, p, i32, i32, p, p]
            lib.oracle_kmeans.argtypes = [p, i64, i32, i32, i32, p, i32, p, p, p]
            for f in (lib.oracle_knn, lib.oracle_knn_probed, lib.oracle_assign, lib.oracle_kmeans):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def knn(x, q, k: int, metric: str = "l2", threads: int | None = None):
    """Exact top-k by FP64 brute force (Sec. 2.1). Returns (dist float64 [nq][k],
    idx int64 [nq][k]); rows padded with (+inf, -1) (-inf for IP) when n < k."""
    x, q = _f32(x), _f32(q)
    n, d = x.shape
    nq = q.shape[0]
    assert q.shape[1] == d
    dist = np.empty((nq, k), np.float64)
    idx = np.empty((nq, k), np.int64)
    rc = _load().oracle_knn(x.ctypes.data, n, d, q.ctypes.data, nq, k, METRICS[metric],
                            threads or default_threads(), dist.ctypes.data, idx.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_knn failed ({rc})")
    return dist, idx


def knn_probed(x, q, k: int, assign, centroids, nprobe: int, metric: str = "l2",
               threads: int | None = None):
    """Exact top-k restricted to the nprobe buckets nearest each query."""
    x, q, centroids = _f32(x), _f32(q), _f32(centroids)
    assign = np.ascontiguousarray(assign, dtype=np.int32)
    n, d = x.shape
    nq = q.shape[0]
    dist = np.empty((nq, k), np.float64)
    idx = np.empty((nq, k), np.int64)
    rc = _load().oracle_knn_probed(x.ctypes.data, n, d, q.ctypes.data, nq, k, METRICS[metric],
                                   assign.ctypes.data, centroids.ctypes.data, centroids.shape[0],
                                   nprobe, threads or default_threads(), dist.ctypes.data, idx.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_knn_probed failed ({rc})")
    return dist, idx


def assign(x, centroids, threads: int | None = None):
    """Nearest centroid (L2, FP64; ties to the lower centroid id)."""
    x, centroids = _f32(x), _f32(centroids)
    n, d = x.shape
    a = np.empty(n, np.int32)
    dd = np.empty(n, np.float64)
    rc = _load().oracle_assign(x.ctypes.data, n, d, centroids.ctypes.data, centroids.shape[0],
                               threads or default_threads(), a.ctypes.data, dd.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_assign failed ({rc})")
    return a, dd


def kmeans(x, init_centroids, iters: int, threads: int | None = None):
    """Lloyd's algorithm in FP64 from the given initial centroids.
    Returns (centroids float64, assignment int32, objective per iteration)."""
    x, init_centroids = _f32(x), _f32(init_centroids)
    n, d = x.shape
    nlist = init_centroids.shape[0]
    c = np.empty((nlist, d), np.float64)
    a = np.empty(n, np.int32)
    obj = np.empty(iters + 1, np.float64)
    rc = _load().oracle_kmeans(x.ctypes.data, n, d, nlist, iters, init_centroids.ctypes.data,
                               threads or default_threads(), c.ctypes.data, a.ctypes.data, obj.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_kmeans failed ({rc})")
    return c, a, obj


def recall_at_k(truth_idx, found_idx) -> float:
    """recall@k = |R cap R_hat| / k averaged over queries (Sec. 2.1)."""
    truth_idx = np.asarray(truth_idx)
    found_idx = np.asarray(found_idx)
    k = truth_idx.shape[1]
    tot = 0
    for t, f in zip(truth_idx, found_idx):
        tot += len(set(t.tolist()) & set(int(v) for v in f if v >= 0))
    return tot / (k * truth_idx.shape[0])


def pair_distances(x, q, ids, metric: str = "l2"):
    """delta(x[ids[r, c]], q[r]) in FP64 (Sec. 2.1); nan where ids < 0."""
    x = np.asarray(x, np.float32)
    q = np.asarray(q, np.float32)
    ids = np.asarray(ids, np.int64)
    out = np.full(ids.shape, np.nan)
    for r in range(ids.shape[0]):
        sel = ids[r] >= 0
        v = x[ids[r][sel]].astype(np.float64)
        qq = q[r].astype(np.float64)
        if metric == "l2":
            out[r, sel] = ((v - qq) ** 2).sum(axis=1)
        elif metric == "ip":
            out[r, sel] = (v * qq).sum(axis=1)
        else:
            out[r, sel] = np.abs(v - qq).sum(axis=1)
    return out
