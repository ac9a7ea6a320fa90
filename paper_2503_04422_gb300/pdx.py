"""Thin Python binding of libpdx (include/pdx.h), argument marshalling only.

Every call goes straight to the C ABI of the same name; all of the search runs
in the library's CUDA kernels. Inputs may be torch tensors (CUDA or CPU) or
numpy arrays: device tensors are passed as device pointers (asynchronous on
the current torch stream), CPU data as host pointers (the library copies it
and synchronises). If the shared library is missing this module raises; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpdx.so")

PDX_OK, PDX_ERR_ARG, PDX_ERR_OOM, PDX_ERR_CUDA, PDX_ERR_TIMEOUT, PDX_ERR_UNSUPPORTED = range(6)
METRIC = {"l2": 0, "ip": 1, "l1": 2}
DTYPE = {"f32": 0, "bf16": 1, "fp8": 2}
PRUNER = {"none": 0, "bond": 1, "ads": 2, "adsampling": 2, "bsa": 3, "ads_bond": 4, "cs_ip": 5}
ORDER = {"dist_to_means": 0, "decreasing": 1, "sequential": 2, "learned": 3}
MEANS = {"block": 0, "collection": 1, "auto": 2}
ENGINE = {"auto": 0, "scan": 1, "tensor": 2}
LAYOUT = {"pdx": 0, "pdx_kernel": 1, "nary": 2, "nary_gather": 3, "dsm": 4}
ARRAY = {"blocks": 0, "ids": 1, "part_blocks": 2, "means": 3, "centroids": 4, "assign": 5, "rotation": 6,
         "variances": 7, "blocks_lp": 8, "scales": 9, "rows": 10}
PHASES = ("preprocess", "find_buckets", "start", "scan", "merge")
STATUS_NAMES = {0: "PDX_OK", 1: "PDX_ERR_ARG", 2: "PDX_ERR_OOM", 3: "PDX_ERR_CUDA", 4: "PDX_ERR_TIMEOUT",
                5: "PDX_ERR_UNSUPPORTED"}


class pdx_build_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("metric", ctypes.c_int), ("storage", ctypes.c_int),
                ("partition_size", ctypes.c_uint32), ("keep_rows", ctypes.c_int32),
                ("dense_rows", ctypes.c_int32), ("keep_dsm", ctypes.c_int32), ("start_clusters", ctypes.c_int32),
                ("cs_first_step", ctypes.c_int32)]


class pdx_ivf_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("base", pdx_build_opts), ("nlist", ctypes.c_uint32),
                ("kmeans_iters", ctypes.c_uint32), ("kmeans_sample", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("transform", ctypes.c_int), ("rotation", ctypes.c_void_p), ("init_centroids", ctypes.c_void_p),
                ("rotation_seed", ctypes.c_uint64)]


class pdx_search_stats(ctypes.Structure):
    _fields_ = [("values_visited", ctypes.c_uint64), ("vectors_scanned", ctypes.c_uint64),
                ("vectors_pruned", ctypes.c_uint64), ("prune_phase_blocks", ctypes.c_uint64),
                ("candidates", ctypes.c_uint64), ("work_items", ctypes.c_uint64),
                ("start_values", ctypes.c_uint64), ("bytes_logical", ctypes.c_uint64),
                ("dense_fallbacks", ctypes.c_uint64), ("phase_ns", ctypes.c_uint64 * 5),
                ("reserved", ctypes.c_uint64 * 2)]
    FIELDS = ("values_visited", "vectors_scanned", "vectors_pruned", "prune_phase_blocks", "candidates",
              "work_items", "start_values", "bytes_logical", "dense_fallbacks")

    def as_dict(self):
        d = {f: int(getattr(self, f)) for f in self.FIELDS}
        d["phase_ns"] = {name: int(v) for name, v in zip(PHASES, self.phase_ns)}
        return d


class pdx_search_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("pruner", ctypes.c_int), ("order", ctypes.c_int),
                ("zone_dims", ctypes.c_uint32), ("selection_threshold", ctypes.c_float), ("eps0", ctypes.c_float),
                ("bsa_m", ctypes.c_float), ("first_step", ctypes.c_uint32), ("start_vectors", ctypes.c_uint32),
                ("blocks_per_item", ctypes.c_uint32), ("stats_out", ctypes.POINTER(pdx_search_stats)),
                ("stats_device", ctypes.c_void_p), ("scan_event_start", ctypes.c_void_p),
                ("scan_event_stop", ctypes.c_void_p), ("means_scope", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_uint32), ("mlp", ctypes.c_void_p), ("mlp_centroids", ctypes.c_void_p),
                ("mlp_ncentroids", ctypes.c_int32), ("engine", ctypes.c_int), ("tau_init", ctypes.c_void_p),
                ("tau_fixed", ctypes.c_int32), ("layout", ctypes.c_int), ("finished_log", ctypes.c_void_p),
                ("finished_count", ctypes.c_void_p), ("finished_cap", ctypes.c_uint64)]


class pdx_index_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("nparts", ctypes.c_int32), ("nblocks", ctypes.c_int64),
                ("metric", ctypes.c_int), ("storage", ctypes.c_int), ("is_ivf", ctypes.c_int32),
                ("unit_norm", ctypes.c_int32), ("device_bytes", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libpdx (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libpdx is not built ({LIB_PATH} missing); run "
                                   "paper_2503_04422_gb300.build.build() first")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
            L.pdx_build_layout.argtypes = [vp, i64, i32, ctypes.POINTER(pdx_build_opts), vp, ctypes.POINTER(vp)]
            L.pdx_ivf_build.argtypes = [vp, i64, i32, ctypes.POINTER(pdx_ivf_opts), vp, ctypes.POINTER(vp)]
            L.pdx_search_exact.argtypes = [vp, vp, i64, i32, ctypes.POINTER(pdx_search_opts), vp, vp, vp]
            L.pdx_search_ivf.argtypes = [vp, vp, i64, i32, i32, ctypes.POINTER(pdx_search_opts), vp, vp, vp]
            L.pdx_free.argtypes = [vp]
            L.pdx_free.restype = None
            L.pdx_kernel_launches.restype = ctypes.c_uint64
            L.pdx_kernel_launches.argtypes = []
            L.pdx_last_error.restype = ctypes.c_char_p
            L.pdx_last_error.argtypes = []
            L.pdx_index_info_get.argtypes = [vp, ctypes.POINTER(pdx_index_info)]
            L.pdx_index_copy_out.argtypes = [vp, ctypes.c_int, vp, sz]
            L.pdx_default_build_opts.argtypes = [ctypes.POINTER(pdx_build_opts)]
            L.pdx_default_ivf_opts.argtypes = [ctypes.POINTER(pdx_ivf_opts)]
            L.pdx_default_search_opts.argtypes = [ctypes.POINTER(pdx_search_opts)]
            for f in ("pdx_default_build_opts", "pdx_default_ivf_opts", "pdx_default_search_opts"):
                getattr(L, f).restype = None
            for f in ("pdx_build_layout", "pdx_ivf_build", "pdx_search_exact", "pdx_search_ivf",
                      "pdx_index_info_get", "pdx_index_copy_out"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


class PdxError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().pdx_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def _check(status: int, where: str):
    if status != PDX_OK:
        raise PdxError(status, where)


def pdx_kernel_launches() -> int:
    return int(lib().pdx_kernel_launches())


def pdx_last_error() -> str:
    return lib().pdx_last_error().decode(errors="replace")


# ---------------------------------------------------------------- marshalling
def _is_torch(a):
    try:
        import torch
        return isinstance(a, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _ptr_f32(a, name):
    """(pointer, keepalive, is_cuda, shape) of a float32 C-contiguous array."""
    if _is_torch(a):
        import torch
        if a.dtype != torch.float32:
            raise TypeError(f"{name} must be float32")
        a = a.contiguous()
        return a.data_ptr(), a, a.is_cuda, tuple(a.shape)
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a.ctypes.data, a, False, a.shape


def _stream(is_cuda, stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if is_cuda:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


class Index:
    """Owns a pdx_index*; freed with pdx_free when garbage collected."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle

    @property
    def info(self) -> pdx_index_info:
        inf = pdx_index_info()
        _check(lib().pdx_index_info_get(self.handle, ctypes.byref(inf)), "pdx_index_info_get")
        return inf

    def copy_out(self, which: str):
        inf = self.info
        shapes = {
            "blocks": ((inf.nblocks, inf.d, 64), np.float32), "ids": ((inf.nblocks * 64,), np.int32),
            "part_blocks": ((inf.nparts + 1,), np.int32), "means": ((inf.nparts, inf.d), np.float32),
            "centroids": ((inf.nparts, inf.d), np.float32), "assign": ((inf.n,), np.int32),
            "rotation": ((inf.d, inf.d), np.float32), "variances": ((inf.d,), np.float32),
            "blocks_lp": ((inf.nblocks, inf.d, 64), np.uint16 if inf.storage == 1 else np.uint8),
            "scales": ((inf.d,), np.float32), "rows": ((inf.n, inf.d), np.float32)}
        shape, dt = shapes[which]
        out = np.empty(shape, dt)
        _check(lib().pdx_index_copy_out(self.handle, ARRAY[which], out.ctypes.data, out.nbytes), "pdx_index_copy_out")
        return out

    def free(self):
        if self.handle:
            lib().pdx_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_opts(metric="l2", storage="f32", partition_size=10000, keep_rows=True,
               dense_rows=False, keep_dsm=False, start_clusters=0, cs_first_step=0) -> pdx_build_opts:
    o = pdx_build_opts()
    lib().pdx_default_build_opts(ctypes.byref(o))
    o.metric = METRIC[metric]
    o.storage = DTYPE[storage]
    o.partition_size = partition_size
    o.keep_rows = int(bool(keep_rows))
    o.dense_rows = int(bool(dense_rows))
    o.keep_dsm = int(bool(keep_dsm))
    o.start_clusters = int(start_clusters)
    o.cs_first_step = int(cs_first_step)
    return o


def search_opts(pruner="bond", order="dist_to_means", zone_dims=None, selection_threshold=None, eps0=None,
                bsa_m=None, first_step=None, start_vectors=None, blocks_per_item=None,
                means_scope=None, ctas_per_sm=None, mlp=None, mlp_centroids=None,
                engine="auto", tau_init=None, tau_fixed=False, layout="pdx", finished_log=None,
                finished_count=None) -> pdx_search_opts:
    """Search options; tau_init (float32 [nq], host or device) seeds each
    query's threshold and tau_fixed keeps it fixed (see include/pdx.h).
    finished_log (int64 device tensor) and finished_count (one-element int64
    device tensor, zeroed by the caller) receive (query << 32) | id of every
    vector the scan carried through all dimensions. The returned struct keeps
    references to these tensors."""
    o = pdx_search_opts()
    lib().pdx_default_search_opts(ctypes.byref(o))
    if tau_init is not None:
        tp, tk, _, _ = _ptr_f32(tau_init, "tau_init")
        o.tau_init = tp
        o._tau_keep = tk
    o.tau_fixed = int(bool(tau_fixed))
    o.layout = LAYOUT[layout]
    if finished_log is not None:
        if finished_count is None or not finished_log.is_cuda or not finished_count.is_cuda:
            raise ValueError("finished_log and finished_count must be CUDA tensors")
        o.finished_log = finished_log.data_ptr()
        o.finished_count = finished_count.data_ptr()
        o.finished_cap = finished_log.numel()
        o._fin_keep = (finished_log, finished_count)
    o.pruner = PRUNER[pruner]
    o.order = ORDER[order]
    o.engine = ENGINE[engine]
    if mlp is not None:
        o.mlp = mlp.handle.value if hasattr(mlp.handle, "value") else mlp.handle
        o.mlp_centroids = mlp_centroids.data_ptr()
        o.mlp_ncentroids = mlp_centroids.shape[0]
    if means_scope is not None:
        o.means_scope = MEANS[means_scope]
    for name, v in (("zone_dims", zone_dims), ("selection_threshold", selection_threshold), ("eps0", eps0),
                    ("bsa_m", bsa_m), ("first_step", first_step), ("start_vectors", start_vectors),
                    ("blocks_per_item", blocks_per_item), ("ctas_per_sm", ctas_per_sm)):
        if v is not None:
            setattr(o, name, v)
    return o


def pdx_build_layout(x, metric="l2", partition_size=10000, storage="f32", stream=None,
                     dense_rows=False, keep_dsm=False, keep_rows=True, start_clusters=0,
                     cs_first_step=0) -> Index:
    """Exact-search index over x [n][d] (Sec. 3, Sec. 6.6); dense_rows also
    keeps the row-major FP32 vectors the tensor-core engine reads, keep_dsm a
    fully dimension-major copy for the DSM layout scan, cs_first_step (inner
    product) the norms the Cauchy-Schwarz pruner "cs_ip" reads."""
    p, keep, cuda, shape = _ptr_f32(x, "x")
    if len(shape) != 2:
        raise ValueError("x must be [n][d]")
    h = ctypes.c_void_p()
    o = build_opts(metric, storage, partition_size, keep_rows=keep_rows, dense_rows=dense_rows, keep_dsm=keep_dsm,
                   start_clusters=start_clusters, cs_first_step=cs_first_step)
    _check(lib().pdx_build_layout(p, shape[0], shape[1], ctypes.byref(o), _stream(cuda, stream), ctypes.byref(h)),
           "pdx_build_layout")
    del keep
    return Index(h)


def pdx_ivf_build(x, nlist, metric="l2", kmeans_iters=10, kmeans_sample=0, seed=2503, transform="none",
                  rotation=None, init_centroids=None, storage="f32", stream=None, rotation_seed=2503,
                  keep_rows=True) -> Index:
    """IVF index whose buckets are PDX blocks (Sec. 2.1, Fig. 2). ADSampling
    rotates by `rotation` when given, else by the library's seeded random
    orthogonal matrix (rotation_seed)."""
    p, keep, cuda, shape = _ptr_f32(x, "x")
    o = pdx_ivf_opts()
    lib().pdx_default_ivf_opts(ctypes.byref(o))
    o.base = build_opts(metric, storage, keep_rows=keep_rows)
    o.rotation_seed = rotation_seed
    o.nlist = nlist
    o.kmeans_iters = kmeans_iters
    o.kmeans_sample = kmeans_sample
    o.seed = seed
    o.transform = PRUNER[transform]
    keeps = [keep]
    if rotation is not None:
        rp, rk, _, _ = _ptr_f32(rotation, "rotation")
        o.rotation = rp
        keeps.append(rk)
    if init_centroids is not None:
        cp, ck, _, _ = _ptr_f32(init_centroids, "init_centroids")
        o.init_centroids = cp
        keeps.append(ck)
    h = ctypes.c_void_p()
    _check(lib().pdx_ivf_build(p, shape[0], shape[1], ctypes.byref(o), _stream(cuda, stream), ctypes.byref(h)),
           "pdx_ivf_build")
    del keeps
    return Index(h)


def _outputs(nq, k, cuda, out):
    if out is not None:
        return out
    if cuda:
        import torch
        return (torch.empty((nq, k), dtype=torch.float32, device="cuda"),
                torch.empty((nq, k), dtype=torch.int64, device="cuda"))
    return np.empty((nq, k), np.float32), np.empty((nq, k), np.int64)


def _out_ptr(a):
    return a.data_ptr() if _is_torch(a) else a.ctypes.data


def pdx_search_exact(index: Index, q, k: int, opts: pdx_search_opts | None = None, out=None, stream=None,
                     stats: bool = False, **kw):
    """Exact k-NN (Sec. 2.1) with PDXearch + PDX-BOND (Sec. 4-5).
    Returns (dist [nq][k], idx [nq][k]) and, with stats=True, a dict of counters."""
    p, keep, cuda, shape = _ptr_f32(q, "q")
    nq = shape[0]
    o = opts if opts is not None else search_opts(**kw)
    st = pdx_search_stats()
    if stats:
        o.stats_out = ctypes.pointer(st)
    od, oi = _outputs(nq, k, cuda, out)
    rc = lib().pdx_search_exact(index.handle, p, nq, k, ctypes.byref(o), _out_ptr(od), _out_ptr(oi),
                                _stream(cuda, stream))
    if stats:
        o.stats_out = None
    _check(rc, "pdx_search_exact")
    del keep
    return (od, oi, st.as_dict()) if stats else (od, oi)


def pdx_search_ivf(index: Index, q, k: int, nprobe: int, opts: pdx_search_opts | None = None, out=None,
                   stream=None, stats: bool = False, **kw):
    """Approximate k-NN over an IVF index with PDXearch (Sec. 4)."""
    p, keep, cuda, shape = _ptr_f32(q, "q")
    nq = shape[0]
    o = opts if opts is not None else search_opts(**kw)
    st = pdx_search_stats()
    if stats:
        o.stats_out = ctypes.pointer(st)
    od, oi = _outputs(nq, k, cuda, out)
    rc = lib().pdx_search_ivf(index.handle, p, nq, k, nprobe, ctypes.byref(o), _out_ptr(od), _out_ptr(oi),
                              _stream(cuda, stream))
    if stats:
        o.stats_out = None
    _check(rc, "pdx_search_ivf")
    del keep
    return (od, oi, st.as_dict()) if stats else (od, oi)


def pdx_merge_topk(dist, idx, metric="l2", out=None, stream=None):
    """Merge per-shard top-k lists dist/idx [nshards][nq][k] (global ids) into
    [nq][k] (pdx_merge_topk). Host arrays merge on the CPU, CUDA tensors on
    the GPU."""
    L = lib()
    f = L.pdx_merge_topk
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    p, keep, cuda, shape = _ptr_f32(dist, "dist")
    if len(shape) != 3:
        raise ValueError("dist must be [nshards][nq][k]")
    ns, nq, k = shape
    if _is_torch(idx):
        import torch
        idx = idx.to(torch.int64).contiguous()
        pi = idx.data_ptr()
    else:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        pi = idx.ctypes.data
    od, oi = _outputs(nq, k, cuda, out)
    _check(f(p, pi, ns, nq, k, METRIC[metric], _out_ptr(od), _out_ptr(oi), _stream(cuda, stream)), "pdx_merge_topk")
    del keep
    return od, oi


def pdx_free(index: Index):
    index.free()


def pdx_search_exact_noalloc(index: Index, q, k: int, opts: pdx_search_opts | None = None, out=None,
                             stream=None, **kw):
    """pdx_search_exact with its scratch in the library's static 32 MiB device
    array (no allocation during the call). q and the outputs must be CUDA
    tensors; overlapping calls on one device race on the shared array."""
    L = lib()
    f = L.pdx_search_exact_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                  ctypes.POINTER(pdx_search_opts), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    p, keep, cuda, shape = _ptr_f32(q, "q")
    nq = shape[0]
    o = opts if opts is not None else search_opts(**kw)
    od, oi = _outputs(nq, k, cuda, out)
    _check(f(index.handle, p, nq, k, ctypes.byref(o), _out_ptr(od), _out_ptr(oi), _stream(cuda, stream)),
           "pdx_search_exact_noalloc")
    del keep
    return od, oi


# ---------------------------------------------------------------- serving
class pdx_server_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("k", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("autotune", ctypes.c_int32), ("tune_cache", ctypes.c_char_p),
                ("search", pdx_search_opts)]


class pdx_server_info_t(ctypes.Structure):
    _fields_ = [("collections", ctypes.c_int32), ("max_bucket", ctypes.c_int32), ("workspace_bytes", ctypes.c_uint64),
                ("graph_launches", ctypes.c_uint64), ("direct_launches", ctypes.c_uint64), ("tunings", ctypes.c_uint64),
                ("entries_ready", ctypes.c_int32)]


def _server_lib():
    L = lib()
    if not getattr(L, "_server_ready", False):
        vp = ctypes.c_void_p
        L.pdx_default_server_opts.argtypes = [ctypes.POINTER(pdx_server_opts)]
        L.pdx_default_server_opts.restype = None
        L.pdx_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, ctypes.POINTER(pdx_server_opts),
                                        ctypes.POINTER(vp)]
        L.pdx_server_create.restype = ctypes.c_int
        L.pdx_server_search.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_int64, vp, vp, vp]
        L.pdx_server_search.restype = ctypes.c_int
        L.pdx_server_info.argtypes = [vp, ctypes.POINTER(pdx_server_info_t)]
        L.pdx_server_info.restype = ctypes.c_int
        L.pdx_server_free.argtypes = [vp]
        L.pdx_server_free.restype = None
        L._server_ready = True
    return L


class Server:
    """Batched exact search over several collections (pdx_server_*)."""

    def __init__(self, indexes, k=10, max_batch=4096, use_graphs=True, autotune=True, tune_cache=None, **search_kw):
        L = _server_lib()
        o = pdx_server_opts()
        L.pdx_default_server_opts(ctypes.byref(o))
        o.k, o.max_batch, o.use_graphs, o.autotune = k, max_batch, int(use_graphs), int(autotune)
        self._cache = tune_cache.encode() if tune_cache else None
        o.tune_cache = self._cache
        o.search = search_opts(**search_kw)
        self.indexes = list(indexes)          # keep the indexes alive
        self.k = k
        arr = (ctypes.c_void_p * len(self.indexes))(*[ix.handle.value if hasattr(ix.handle, "value") else ix.handle
                                                      for ix in self.indexes])
        h = ctypes.c_void_p()
        _check(L.pdx_server_create(arr, len(self.indexes), ctypes.byref(o), ctypes.byref(h)), "pdx_server_create")
        self.handle = h

    def search(self, collection: int, q, out=None, stream=None):
        L = _server_lib()
        p, keep, cuda, shape = _ptr_f32(q, "q")
        od, oi = _outputs(shape[0], self.k, cuda, out)
        _check(L.pdx_server_search(self.handle, collection, p, shape[0], _out_ptr(od), _out_ptr(oi),
                                   _stream(cuda, stream)), "pdx_server_search")
        del keep
        return od, oi

    @property
    def info(self):
        inf = pdx_server_info_t()
        _check(_server_lib().pdx_server_info(self.handle, ctypes.byref(inf)), "pdx_server_info")
        return {f: getattr(inf, f) for f, _ in inf._fields_}

    def free(self):
        if self.handle:
            _server_lib().pdx_server_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------- order network
def _mlp_lib():
    L = lib()
    if not getattr(L, "_mlp_ready", False):
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.pdx_mlp_create.argtypes = [i32, i32, ctypes.c_uint64, ctypes.POINTER(vp)]
        L.pdx_mlp_free.argtypes = [vp]
        L.pdx_mlp_free.restype = None
        L.pdx_mlp_param_count.argtypes = [vp]
        L.pdx_mlp_param_count.restype = ctypes.c_size_t
        L.pdx_mlp_set_params.argtypes = [vp, vp, ctypes.c_size_t]
        L.pdx_mlp_get_params.argtypes = [vp, vp, ctypes.c_size_t]
        L.pdx_mlp_forward.argtypes = [vp, vp, i64, i32, vp, vp]
        L.pdx_mlp_backward.argtypes = [vp, vp, vp, i64, vp, ctypes.POINTER(ctypes.c_float), vp]
        L.pdx_mlp_train.argtypes = [vp, vp, vp, i64, i32, i32, ctypes.c_float, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_float), vp]
        L.pdx_order_targets.argtypes = [vp, vp, i64, vp, i32, vp, vp]
        L.pdx_mlp_inputs.argtypes = [vp, i64, i32, vp, i32, vp, vp]
        L.pdx_mlp_inputs.restype = ctypes.c_int
        for f in ("pdx_mlp_create", "pdx_mlp_set_params", "pdx_mlp_get_params", "pdx_mlp_forward",
                  "pdx_mlp_backward", "pdx_mlp_train", "pdx_order_targets"):
            getattr(L, f).restype = ctypes.c_int
        L._mlp_ready = True
    return L


class Mlp:
    """Order-proposal network (pdx_mlp_*). Device tensors in, device tensors out."""

    def __init__(self, d, hidden=256, seed=2503):
        L = _mlp_lib()
        h = ctypes.c_void_p()
        _check(L.pdx_mlp_create(d, hidden, seed, ctypes.byref(h)), "pdx_mlp_create")
        self.handle, self.d, self.hidden = h, d, hidden
        self.count = int(L.pdx_mlp_param_count(h))

    def get_params(self):
        out = np.empty(self.count, np.float32)
        _check(_mlp_lib().pdx_mlp_get_params(self.handle, out.ctypes.data, self.count), "pdx_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        _check(_mlp_lib().pdx_mlp_set_params(self.handle, p.ctypes.data, p.size), "pdx_mlp_set_params")

    def forward(self, u, bf16=False):
        import torch
        y = torch.empty((u.shape[0], self.d), dtype=torch.float32, device=u.device)
        _check(_mlp_lib().pdx_mlp_forward(self.handle, u.data_ptr(), u.shape[0], int(bf16), y.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream), "pdx_mlp_forward")
        return y

    def backward(self, u, t):
        import torch
        g = np.empty(self.count, np.float32)
        loss = ctypes.c_float()
        _check(_mlp_lib().pdx_mlp_backward(self.handle, u.data_ptr(), t.data_ptr(), u.shape[0], g.ctypes.data,
                                           ctypes.byref(loss), torch.cuda.current_stream().cuda_stream),
               "pdx_mlp_backward")
        return g, loss.value

    def train(self, u, t, epochs=10, batch=256, lr=1e-3, seed=1):
        import torch
        loss = ctypes.c_float()
        _check(_mlp_lib().pdx_mlp_train(self.handle, u.data_ptr(), t.data_ptr(), u.shape[0], epochs, batch, lr, seed,
                                        ctypes.byref(loss), torch.cuda.current_stream().cuda_stream), "pdx_mlp_train")
        return loss.value

    def free(self):
        if self.handle:
            _mlp_lib().pdx_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def pdx_order_targets(index: Index, q, ids, m=None):
    """Trace targets for the network (see pdx.h), q and ids CUDA tensors."""
    import torch
    m = ids.shape[1] if m is None else m
    t = torch.empty((q.shape[0], index.info.d), dtype=torch.float32, device=q.device)
    _check(_mlp_lib().pdx_order_targets(index.handle, q.data_ptr(), q.shape[0], ids.data_ptr(), m, t.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream), "pdx_order_targets")
    return t


def pdx_mlp_inputs(q, centroids):
    """[q; nearest centroid] rows for the network (CUDA tensors)."""
    import torch
    u = torch.empty((q.shape[0], 2 * q.shape[1]), dtype=torch.float32, device=q.device)
    _check(_mlp_lib().pdx_mlp_inputs(q.data_ptr(), q.shape[0], q.shape[1], centroids.data_ptr(), centroids.shape[0],
                                     u.data_ptr(), torch.cuda.current_stream().cuda_stream), "pdx_mlp_inputs")
    return u
