#!/usr/bin/env python
"""Throughput of the PDX exact search (PDXearch + PDX-BOND) on GB300.

A step is one exact top-10 search of the whole query batch (1,000 queries)
over the 1M x 768 Gaussian-mixture collection, inputs resident in HBM. The
JSON line reports queries/s, the roofline of the dominant kernel (the PDXearch
scan) from live CUDA events and the kernel's own counters, the end-to-end
rate through the C ABI with host buffers, the CPU oracle on the host cores,
and the SM clocks seen during the timed region.

Usage: python bench.py [--gpus N --steps K --warmup W --impl ours|reference]
For N > 1 launch under torchrun: every rank holds a replica of the
collection and searches its own batch of queries (weak scaling, no
collective on the data path). With --shard the collection is split by id
range instead: every rank answers the same queries over its shard, and the
per-shard top-k lists are all-gathered over NCCL and merged on the device
(strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("queries/sec at exact top-10 (and recall@10=0.95 IVF); HBM GB/s vs peak; learned vs plain")
WORKLOADS = {
    "bond_exact_1m_d768": dict(k=10, pruner="bond"),
    "plain_scan_10k_d128": dict(k=10, pruner="none"),
    "ivf_1m_d960": dict(k=10, pruner="ads", nlist=1024),
    "learned_order_2m_d1536": dict(k=10, pruner="bond", metric="ip", nclusters=1024, traces=50_000),
    "serving_64_fp8": dict(k=100, pruner="bond", storage="fp8", batches=1000, max_batch=4096),
    "serving_batch1_fp8": dict(k=100, pruner="bond", storage="fp8"),
    "layouts": dict(k=10),
    "mips_1m_d768": dict(k=10, pruner="cs_ip", metric="ip"),
}
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in the background."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


SCAN_SOURCES = ("pdx_search.cu", "pdx_internal.cuh")
DENSE_SOURCES = ("pdx_dense.cu", "pdx_internal.cuh")


def _kernel_hash(sources=SCAN_SOURCES):
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2503_04422_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_per_launch(key):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    try:
        with open(PROFILE_TRAFFIC) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    e = t.get(key)
    sources = DENSE_SOURCES if key.endswith(":tensor") else SCAN_SOURCES
    if not e or e.get("kernel_hash") != _kernel_hash(sources):
        return None
    return e.get("dram_bytes_per_launch")


def _peak_tf32():
    """TF32 dense tensor peak: the measured BF16 burst peak times the nominal
    TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x 1.1/2.25"
    except (OSError, ValueError, KeyError):
        return 1900.0 * 1.1 / 2.25, "fallback bf16 x 1.1/2.25"


def _peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def cpu_oracle_rate(x, q, k, budget_s=15.0, metric="l2"):
    """FP64 oracle on the host cores over batches of queries until the budget
    is spent. Returns (queries/s, threads, queries done)."""
    from oracle import knn as ok
    threads = ok.default_threads()
    done, t0 = 0, time.perf_counter()
    batch = max(threads, 8)
    while True:
        sel = q[(done % q.shape[0]):(done % q.shape[0]) + batch]
        ok.knn(x, sel, k, metric, threads=threads)
        done += sel.shape[0]
        el = time.perf_counter() - t0
        if el >= budget_s:
            return done / el, threads, done


def run_reference(args, rank, world):
    """The oracle on the host cores: each step searches a bounded sample of the
    same workload (a few queries against the full collection)."""
    if rank != 0:
        return
    import pdx_synth
    from oracle import knn as ok
    ok.build()
    spec = WORKLOADS[args.workload]
    x, q = pdx_synth.make(args.workload)
    threads = ok.default_threads()
    per_step = max(threads, 8)
    for s in range(args.warmup):
        ok.knn(x, q[:per_step], spec["k"], threads=threads)
    t0 = time.perf_counter()
    done = 0
    for s in range(args.steps):
        sel = q[(s * per_step) % q.shape[0]:][:per_step]
        ok.knn(x, sel, spec["k"], threads=threads)
        done += sel.shape[0]
    el = time.perf_counter() - t0
    value = done / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": x.shape[0], "d": x.shape[1], "k": spec["k"],
                       "queries_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} queries per step against all {x.shape[0]} vectors"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _e2e(pdx, ix, q, k, opts, stream, flush, K, world, dist):
    """Same search through the C ABI with pinned host buffers: the call copies
    the queries in and the results out (and synchronises) inside the timed
    region."""
    import torch
    nq, d = q.shape
    q_host = torch.from_numpy(q).pin_memory()
    od_h = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    oi_h = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    opts.scan_event_start = opts.scan_event_stop = opts.stats_device = None
    for _ in range(2):
        pdx.pdx_search_exact(ix, q_host, k, opts=opts, out=(od_h, oi_h), stream=stream.cuda_stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    for i in range(K):
        flush.zero_()
        ev[i][0].record(stream)
        pdx.pdx_search_exact(ix, q_host, k, opts=opts, out=(od_h, oi_h), stream=stream.cuda_stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return {"value": nq * world * K / (ms / 1e3), "unit": "queries/s", "h2d_bytes_per_step": nq * d * 4,
            "d2h_bytes_per_step": nq * k * 12}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import pdx_synth
    from paper_2503_04422_gb300 import build as pbuild
    pbuild.build()
    from paper_2503_04422_gb300 import pdx

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    spec = WORKLOADS[args.workload]
    k = spec["k"]
    base_nq = args.nq or pdx_synth.WORKLOADS[args.workload]["nq"]
    if args.shard:
        # sharded collection: every rank holds the id range [lo, hi) and answers
        # the same queries; the per-shard lists are all-gathered and merged
        from paper_2503_04422_gb300 import shard
        x_all, q_all = pdx_synth.make(args.workload, n=args.n, nq=base_nq)
        q = np.ascontiguousarray(q_all)
        lo, hi = shard.shard_range(x_all.shape[0], rank, world)
        x = np.ascontiguousarray(x_all[lo:hi])
        n_total = x_all.shape[0]
        del x_all
    else:
        x, q_all = pdx_synth.make(args.workload, n=args.n, nq=base_nq * world)
        q = np.ascontiguousarray(q_all[rank * base_nq:(rank + 1) * base_nq])
        lo, n_total = 0, x.shape[0]
    n, d = x.shape
    nq = q.shape[0]
    pruner = args.pruner or spec["pruner"]
    engine = args.engine or ("tensor" if pruner == "none" else "auto")
    tensor = pruner == "none" and engine == "tensor"
    metric = spec.get("metric", "l2")
    ix = pdx.pdx_build_layout(torch.from_numpy(x).cuda(), metric=metric, storage=args.storage, dense_rows=tensor,
                              cs_first_step=4 if pruner == "cs_ip" else 0)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    q_dev = torch.from_numpy(q).cuda()
    od = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    oi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    stats_dev = torch.zeros(16, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    opts = pdx.search_opts(pruner=pruner, engine=engine if pruner == "none" else "auto",
                           first_step=args.first_step, ctas_per_sm=args.ctas_per_sm,
                           start_vectors=args.start_vectors, selection_threshold=args.selection_threshold)
    stream = torch.cuda.current_stream()

    def step(ev_scan=None):
        if ev_scan is not None:
            opts.scan_event_start = ev_scan[0].cuda_event
            opts.scan_event_stop = ev_scan[1].cuda_event
            opts.stats_device = stats_dev.data_ptr()
        else:
            opts.scan_event_start = opts.scan_event_stop = opts.stats_device = None
        pdx.pdx_search_exact(ix, q_dev, k, opts=opts, out=(od, oi))
        if args.shard:   # the exchange step: global ids, NCCL all-gather, device merge
            return shard.gather_merge(od, oi, lo)
        return od, oi

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    ev_scan = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for a, b in ev_scan:          # torch creates event handles lazily: materialise them
        a.record(stream)
        b.record(stream)
    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stats_dev.zero_()
    launches0 = pdx.pdx_kernel_launches()
    clocks.start()
    for i in range(K):
        flush.zero_()                                   # L2 flush between timed steps (not timed)
        ev[i][0].record(stream)
        step(ev_scan[i])
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = pdx.pdx_kernel_launches() - launches0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    scan_ms = [a.elapsed_time(b) for a, b in ev_scan]
    tot_ms = sum(step_ms)
    st = stats_dev.cpu().numpy().astype(np.uint64)
    if dist:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    ms_per_step = tot_ms / K
    # replicas: every rank answers its own queries (weak scaling); shards: all
    # ranks answer the same queries over their part of the collection (strong)
    value = nq * (1 if args.shard else world) * K / (tot_ms / 1e3)

    # roofline of the dominant kernel from its event-timed launches: the
    # PDXearch scan (logical bytes read) or the tensor-core GEMM (2 nq n d FLOP)
    values_per_launch = float(st[0]) / K
    esize = {"f32": 4.0, "bf16": 2.0, "fp8": 1.0}[args.storage]
    # logical bytes of the scan: values visited x element size, plus the FP32
    # rerank rows of low-precision candidates
    bytes_per_launch = values_per_launch * esize + (0.0 if args.storage == "f32" else float(st[4]) / K * d * 4.0)
    scan_avg_ms = sum(scan_ms) / K
    achieved = bytes_per_launch / (scan_avg_ms / 1e3) / 1e9
    peak, peak_kind = _peak_hbm()
    traffic = _traffic_per_launch(args.workload) if args.storage == "f32" else None
    if pruner == "none":
        traffic = None
    if tensor:
        # two launches per step (bound pass, emit pass), each the full product;
        # the event bracket also holds the small per-query select between them
        flop = 2.0 * nq * n * d
        launch_ms = scan_avg_ms / 2.0
        tflops = flop / (launch_ms / 1e3) / 1e12
        tpeak, tkind = _peak_tf32()
        roofline = {"bound": "tensor", "kernel": "dense_tc_kernel<16,L2,*> (tcgen05.mma kind::tf32, TMA, TMEM)",
                    "achieved": tflops, "peak": tpeak, "peak_kind": tkind, "unit": "TFLOP/s",
                    "frac": tflops / tpeak, "traffic": _traffic_per_launch(args.workload + ":tensor"),
                    "algorithmic_flop_per_launch": flop, "launches_per_step": 2,
                    "launch_ms_avg": launch_ms, "bracket": "both GEMM launches and the select between them",
                    "per_unit": {"flop_per_query": 2.0 * n * d, "units_per_launch": nq}}
    else:
        roofline = {"bound": "hbm",
                    "kernel": f"pdxsearch_kernel<{pruner.upper()},{metric.upper()},{args.storage.upper()}>",
                    "achieved": achieved,
                    "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "algorithmic_bytes_per_launch": bytes_per_launch,
                    "scan_ms_avg": scan_avg_ms,
                    # DRAM bytes the kernel really moves (ncu, per launch) over its live duration:
                    # the working set is L2-resident, so this stays far below the logical rate
                    "dram_gbs": (traffic / (scan_avg_ms / 1e3) / 1e9) if traffic else None,
                    "dram_frac": (traffic / (scan_avg_ms / 1e3) / 1e9 / peak) if traffic else None,
                    "per_unit": {"bytes_per_query": bytes_per_launch / nq, "units_per_launch": nq}}

    # end to end through the C ABI with host (pinned) buffers
    e2e = None
    if not args.no_e2e and not args.shard:
        e2e = _e2e(pdx, ix, q, k, opts, stream, flush, K, world, dist)
    elif not args.no_e2e:
        # shards: host queries in, search, exchange, merged results back to the host
        q_host = torch.from_numpy(q).pin_memory()
        rd = torch.empty((nq, k), dtype=torch.float32).pin_memory()
        ri = torch.empty((nq, k), dtype=torch.int64).pin_memory()
        ev_e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        for i in range(K):
            flush.zero_()
            ev_e[i][0].record(stream)
            q_dev.copy_(q_host, non_blocking=True)
            md, mi = step()
            rd.copy_(md, non_blocking=True)
            ri.copy_(mi, non_blocking=True)
            ev_e[i][1].record(stream)
        torch.cuda.synchronize()
        e_ms = sum(a_.elapsed_time(b_) for a_, b_ in ev_e)
        if dist:
            t = torch.tensor([e_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        e2e = {"value": nq * K / (e_ms / 1e3), "unit": "queries/s", "h2d_bytes_per_step": nq * d * 4,
               "d2h_bytes_per_step": nq * k * 12}

    # the other exact engines on the same workload (same exact results): no
    # pruning, q.x on the tensor cores (the L2 decomposition's, or the inner
    # product itself), and for the inner-product pruner also the plain scan
    def time_engine(index, opts_t):
        od_t = torch.empty_like(od)
        oi_t = torch.empty_like(oi)
        for _ in range(args.warmup):
            pdx.pdx_search_exact(index, q_dev, k, opts=opts_t, out=(od_t, oi_t))
        ev_t = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        for i in range(K):
            flush.zero_()
            ev_t[i][0].record(stream)
            pdx.pdx_search_exact(index, q_dev, k, opts=opts_t, out=(od_t, oi_t))
            ev_t[i][1].record(stream)
        torch.cuda.synchronize()
        t_ms = sum(a_.elapsed_time(b_) for a_, b_ in ev_t)
        return t_ms, bool(torch.equal(oi_t, oi))

    alt = None
    plain = None
    if pruner in ("bond", "cs_ip") and args.storage == "f32" and not args.no_alt and not args.shard:
        ix_t = pdx.pdx_build_layout(torch.from_numpy(x).cuda(), metric=metric, dense_rows=True)
        torch.cuda.synchronize()
        t_ms, same = time_engine(ix_t, pdx.search_opts(pruner="none", engine="tensor"))
        alt = {"engine": "tensor (no pruning; TF32 tcgen05 GEMM, proven margins, FP32 rerank)",
               "value": nq * world * K / (t_ms / 1e3), "unit": "queries/s", "ms_per_step": t_ms / K,
               ("same_ids_as_pdx_bond" if pruner == "bond" else "same_ids_as_cs_ip"): same}
        del ix_t
        torch.cuda.empty_cache()
    if pruner == "cs_ip" and not args.no_alt and not args.shard:
        t_ms, same = time_engine(ix, pdx.search_opts(pruner="none", engine="scan"))
        plain = {"engine": "pdx scan, no pruning (inner product)", "value": nq * world * K / (t_ms / 1e3),
                 "unit": "queries/s", "ms_per_step": t_ms / K, "same_ids_as_cs_ip": same}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, thr, done = cpu_oracle_rate(x, q, k, budget_s=args.cpu_budget, metric=metric)
        cpu = {"value": rate, "unit": "queries/s", "cores": thr, "kind": "oracle",
               "sample": f"{done} queries against all {n} vectors, FP64 brute force with full sort"}
    if rank == 0:
        pruned = float(st[2]) / max(1.0, float(st[1]))
        line = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong" if args.shard else "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": args.workload, "n": n_total, "d": d, "nq_per_gpu": nq, "k": k,
                       "storage": args.storage,
                       "parallelism": (f"shard{world}: ids [lo, hi) per rank, NCCL all-gather of the "
                                       "per-shard top-k, pdx_merge_topk on the device") if args.shard
                       else f"replicas{world}: every rank searches its own queries over the whole collection",
                       "pruner": pruner, "engine": "tensor (TF32 GEMM + FP32 rerank)" if tensor else "pdx scan",
                       "metric": metric,
                       "order": "storage order (the stored norms fix it)" if pruner == "cs_ip" else "dist_to_means",
                       "means": "collection (automatic for exact search)", "zone_dims": "1 (automatic)",
                       "first_step": int(opts.first_step), "selection_threshold": round(float(opts.selection_threshold), 3),
                       "start": (f"start clusters: {min(1024, n // 4096)} k-means centroids x 64 member vectors, "
                                 "the 2 nearest per query" if n >= 65536 and pruner not in ("none", "cs_ip")
                                 else f"the first {int(opts.start_vectors)} stored vectors"),
                       "ctas_per_sm": int(opts.ctas_per_sm) or "automatic (4 when four CTAs fit with 32 KB of L1, else 3)",
                       "l2": (f"collection {n * d * 4 / 1e9:.3g} GB; 256 MB L2 flush between timed steps "
                              "(untimed)")},
            "roofline": roofline,
            "pruning": {"values_visited_fraction": values_per_launch / (n * d * nq), "vectors_pruned_fraction": pruned,
                        "candidates_reranked_per_query": float(st[4]) / K / nq,
                        "dense_fallbacks": int(st[8])},
            "e2e": e2e,
            "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / K,
            "clocks": clk,
            "cpu_baseline": cpu,
            "other_exact_engine": alt, "plain_scan": plain,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_ivf(args, rank, world, local_rank):
    """IVF search (Sec. 6.3-6.4 setting): 1M x 960 rotated Gaussian mixture,
    nlist = 1024, 10,000 queries, k = 10. For each pruner the nprobe sweep
    1..128 runs, and the line reports queries/s at the smallest nprobe whose
    recall@10 is >= 0.95. Recall is measured against the FP64 oracle's exact
    top-10 over all N vectors for a subsample of the queries (the CPU-baseline
    leg: the oracle's brute force on the host cores, timed, is both the
    cpu_baseline figure and the ground truth). The line also carries the
    per-phase split of one search at the chosen nprobe (the Table 6
    breakdown: preprocessing, finding buckets, START, scan, merge)."""
    import numpy as np
    import torch

    import pdx_synth
    from paper_2503_04422_gb300 import build as pbuild
    pbuild.build()
    from paper_2503_04422_gb300 import pdx

    torch.cuda.set_device(local_rank)
    spec = WORKLOADS[args.workload]
    k, nlist = spec["k"], spec["nlist"]
    nq = args.nq or pdx_synth.WORKLOADS[args.workload]["nq"]
    x, q = pdx_synth.make(args.workload, n=args.n, nq=nq)
    n, d = x.shape
    xd = torch.from_numpy(x).cuda()
    qd = torch.from_numpy(q).cuda()
    cpu = None
    if not args.no_cpu_baseline:
        # CPU-baseline leg: the FP64 oracle on the host cores over a subsample
        # of the queries; its exact top-10 is the recall ground truth
        from oracle import knn as ok
        ok.build()
        sample = np.linspace(0, nq - 1, num=min(nq, args.recall_queries)).astype(np.int64)
        threads = ok.default_threads()
        t0 = time.perf_counter()
        truth = ok.knn(x, np.ascontiguousarray(q[sample]), k, threads=threads)[1]
        el = time.perf_counter() - t0
        cpu = {"value": sample.size / el, "unit": "queries/s", "cores": threads, "kind": "oracle",
               "sample": f"{sample.size} queries against all {n} vectors, FP64 brute force with full sort "
                         "(also the recall ground truth)"}
        truth_kind = "oracle"
    else:
        exact = pdx.pdx_build_layout(xd)
        truth = pdx.pdx_search_exact(exact, qd, k, pruner="bond")[1].cpu().numpy()
        exact.free()
        torch.cuda.empty_cache()
        sample = np.arange(nq)
        truth_kind = "library exact search (PDX-BOND)"

    def recall_at_k(t, r):
        return float(np.mean([len(set(a.tolist()) & set(b.tolist())) / t.shape[1] for a, b in zip(t, r)]))

    od = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    oi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    stats_dev = torch.zeros(16, dtype=torch.int64, device="cuda")
    results = {}
    pruners = [p.strip() for p in args.pruners.split(",")]
    transforms = {"ads": "ads", "ads_bond": "ads", "bsa": "bsa", "bond": "none", "none": "none"}
    built = {}
    clocks = ClockSampler(local_rank)
    clocks.start()
    for pruner in pruners:
        tr = transforms[pruner]
        if tr not in built:
            t0 = time.perf_counter()
            built[tr] = pdx.pdx_ivf_build(xd, nlist=nlist, kmeans_iters=10, kmeans_sample=min(n, 256 * nlist),
                                          transform=tr, rotation_seed=77, storage=args.storage)
            torch.cuda.synchronize()
            build_s = time.perf_counter() - t0
        ix = built[tr]
        rows = []
        for nprobe in (1, 2, 4, 8, 16, 32, 64, 128):
            opts = pdx.search_opts(pruner=pruner, first_step=args.first_step, ctas_per_sm=args.ctas_per_sm)
            for _ in range(args.warmup):
                pdx.pdx_search_ivf(ix, qd, k, nprobe, opts=opts, out=(od, oi))
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
            for a_, b_ in evs:
                a_.record()
                b_.record()
            stats_dev.zero_()
            torch.cuda.synchronize()
            launches0 = pdx.pdx_kernel_launches()
            for i in range(args.steps):
                opts.scan_event_start, opts.scan_event_stop = evs[i][0].cuda_event, evs[i][1].cuda_event
                opts.stats_device = stats_dev.data_ptr()
                ev[i][0].record()
                pdx.pdx_search_ivf(ix, qd, k, nprobe, opts=opts, out=(od, oi))
                ev[i][1].record()
            torch.cuda.synchronize()
            launches = pdx.pdx_kernel_launches() - launches0
            ms = sum(a_.elapsed_time(b_) for a_, b_ in ev) / args.steps
            scan_ms = sum(a_.elapsed_time(b_) for a_, b_ in evs) / args.steps
            st = stats_dev.cpu().numpy().astype(np.float64)
            rec = recall_at_k(truth, oi.cpu().numpy()[sample])
            esize = {"f32": 4.0, "bf16": 2.0, "fp8": 1.0}[args.storage]
            byts = st[0] / args.steps * esize + (0.0 if args.storage == "f32" else st[4] / args.steps * d * 4.0)
            rows.append(dict(nprobe=nprobe, qps=nq / (ms / 1e3), ms=ms, recall=rec, scan_ms=scan_ms,
                             scan_gbs=byts / (scan_ms / 1e3) / 1e9, gpu_launches=int(launches),
                             visited_fraction=st[0] / args.steps / (nq * nprobe * (n / nlist) * d)))
            print(json.dumps({"pruner": pruner, **rows[-1]}), file=sys.stderr, flush=True)
        ok_rows = [r for r in rows if r["recall"] >= 0.95]
        chosen = ok_rows[0] if ok_rows else None
        if chosen is not None:
            # per-phase device time of one search at this nprobe (Table 6)
            o1 = pdx.search_opts(pruner=pruner, first_step=args.first_step, ctas_per_sm=args.ctas_per_sm)
            _, _, st1 = pdx.pdx_search_ivf(ix, qd, k, chosen["nprobe"], opts=o1, out=(od, oi), stats=True)
            ph = st1["phase_ns"]
            tot = max(1, sum(ph.values()))
            chosen["phases_ms"] = {p: v / 1e6 for p, v in ph.items()}
            chosen["phases_share"] = {p: v / tot for p, v in ph.items()}
        results[pruner] = dict(at_recall_095=chosen, sweep=rows)
    clk = clocks.stop()
    main_p = pruners[0]
    best = results[main_p]["at_recall_095"] or results[main_p]["sweep"][-1]
    peak, peak_kind = _peak_hbm()
    line = {"metric": METRIC, "value": best["qps"], "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "d": d, "nq": nq, "k": k, "nlist": nlist,
                       "pruner": main_p, "storage": args.storage, "nprobe": best["nprobe"],
                       "recall@10": best["recall"], "recall_queries": int(sample.size), "recall_truth": truth_kind,
                       "rotation": "library-drawn Haar orthogonal (rotation_seed 77)",
                       "l2": "collection 3.8 GB > L2"},
            "roofline": {"bound": "hbm", "kernel": f"pdxsearch_kernel<{main_p.upper()},L2>", "achieved": best["scan_gbs"],
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": best["scan_gbs"] / peak,
                         "traffic": None},
            "pruners": {p: r["at_recall_095"] for p, r in results.items()},
            "gpu_launches": best["gpu_launches"], "clocks": clk,
            "cpu_baseline": cpu,
            "sweeps": {p: r["sweep"] for p, r in results.items()}}
    print(json.dumps(line), flush=True)


def run_learned(args, rank, world, local_rank):
    """Learned visit order vs the distance-to-means heuristic (exact PDX-BOND,
    inner product on unit-norm 1536-d embeddings). The network [q; c] -> 256 ->
    1536 is trained on the GPU on traces of the plain method for separate
    training queries. The line reports queries/s with the learned order, next to
    the heuristic's, at identical exact results. Following the fallback rule,
    the learned order is used only if it visits at least 1% fewer values than
    the heuristic on a validation split."""
    import numpy as np
    import torch

    import pdx_synth
    from paper_2503_04422_gb300 import build as pbuild
    pbuild.build()
    from paper_2503_04422_gb300 import pdx

    torch.cuda.set_device(local_rank)
    spec = WORKLOADS[args.workload]
    k = spec["k"]
    nq = args.nq or pdx_synth.WORKLOADS[args.workload]["nq"]
    ntr = args.traces or spec["traces"]
    n_full = args.n or pdx_synth.WORKLOADS[args.workload]["n"]
    d = pdx_synth.WORKLOADS[args.workload]["d"]
    t0 = time.perf_counter()
    x, q_all = pdx_synth.embedding_like(n_full, d, nq + ntr + 1000)
    gen_s = time.perf_counter() - t0
    xd = torch.from_numpy(x).cuda()
    del x
    q_all = torch.from_numpy(q_all).cuda()
    q_test, q_tr, q_val = q_all[:nq].contiguous(), q_all[nq:nq + ntr].contiguous(), q_all[nq + ntr:].contiguous()
    ix = pdx.pdx_build_layout(xd, metric="ip")
    # clusters for the network input: k-means on a sample (an IVF index over it)
    nsample = min(n_full, 256 * spec["nclusters"])
    clus = pdx.pdx_ivf_build(xd[:nsample].contiguous(), nlist=spec["nclusters"], kmeans_iters=8)
    cent = torch.from_numpy(clus.copy_out("centroids")).cuda()
    del clus
    torch.cuda.synchronize()
    # traces: the vectors the plain method ranked just behind the top-k, plus
    # a sample of the vectors it pruned
    t0 = time.perf_counter()
    m_hard, m_rand = 48, 160
    tg = []
    for c0 in range(0, ntr, 5000):
        qq = q_tr[c0:c0 + 5000].contiguous()
        _, ids = pdx.pdx_search_exact(ix, qq, k + m_hard)
        rnd = torch.randint(0, n_full, (qq.shape[0], m_rand), device="cuda", dtype=torch.int64,
                            generator=torch.Generator(device="cuda").manual_seed(c0))
        tg.append(pdx.pdx_order_targets(ix, qq, torch.cat([ids[:, k:], rnd], dim=1).contiguous()))
    targets = torch.cat(tg)
    u = pdx.pdx_mlp_inputs(q_tr, cent)
    trace_s = time.perf_counter() - t0
    net = pdx.Mlp(d, 256, seed=2503)
    t0 = time.perf_counter()
    loss = net.train(u, targets, epochs=args.epochs, batch=256, lr=1e-3)
    train_s = time.perf_counter() - t0
    heur = pdx.search_opts(pruner="bond")
    learned = pdx.search_opts(pruner="bond", order="learned", mlp=net, mlp_centroids=cent)
    # the heuristic order is the fallback: the learned one is used only if it
    # visits fewer values on a validation split
    _, iv_h, sv_h = pdx.pdx_search_exact(ix, q_val, k, opts=pdx.search_opts(pruner="bond"), stats=True)
    _, iv_l, sv_l = pdx.pdx_search_exact(ix, q_val, k, opts=pdx.search_opts(pruner="bond", order="learned", mlp=net,
                                                                             mlp_centroids=cent), stats=True)
    # (by at least 1%: the network's inference costs time, and a smaller
    # difference is within what the split itself varies by)
    use_learned = sv_l["values_visited"] < 0.99 * sv_h["values_visited"]
    od = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    oi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    stats_dev = torch.zeros(16, dtype=torch.int64, device="cuda")

    def timed(opts):
        for _ in range(args.warmup):
            pdx.pdx_search_exact(ix, q_test, k, opts=opts, out=(od, oi))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        stats_dev.zero_()
        opts.stats_device = stats_dev.data_ptr()
        torch.cuda.synchronize()
        for a_, b_ in ev:
            a_.record()
            pdx.pdx_search_exact(ix, q_test, k, opts=opts, out=(od, oi))
            b_.record()
        torch.cuda.synchronize()
        opts.stats_device = None
        ms = sum(a_.elapsed_time(b_) for a_, b_ in ev) / args.steps
        st = stats_dev.cpu().numpy().astype(np.float64)
        return ms, st[0] / args.steps / (n_full * d * nq), oi.clone()

    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = pdx.pdx_kernel_launches()
    ms_h, vis_h, res_h = timed(heur)
    l1 = pdx.pdx_kernel_launches()
    ms_l, vis_l, res_l = timed(learned)
    l2 = pdx.pdx_kernel_launches()
    clk = clocks.stop()
    same = bool(torch.equal(res_h, res_l))
    chosen = ms_l if use_learned else ms_h
    line = {"metric": METRIC, "value": nq / (chosen / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": chosen, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n": n_full, "d": d, "nq": nq, "k": k, "metric": "ip (unit norm)",
                       "network": f"{2 * d}-256-{d}, BF16 inference weights", "traces": ntr,
                       "clusters": spec["nclusters"], "epochs": args.epochs},
            "learned_vs_plain": {"learned_qps": nq / (ms_l / 1e3), "plain_qps": nq / (ms_h / 1e3),
                                 "learned_values_visited": vis_l, "plain_values_visited": vis_h,
                                 "identical_results": same, "validation_prefers_learned": bool(use_learned),
                                 "train_loss": loss, "train_s": train_s, "trace_s": trace_s, "gen_s": gen_s},
            # timed() launches the warm-up and the timed steps alike
            "gpu_launches": int(((l2 - l1) if use_learned else (l1 - l0)) * args.steps / (args.steps + args.warmup)),
            "gpu_launches_per_step": ((l2 - l1) if use_learned else (l1 - l0)) / (args.steps + args.warmup),
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_serving(args, rank, world, local_rank):
    """Batched uneven serving: 64 collections (sizes log-uniform 1e4..2e6, D in
    {96, 384, 1024}, Gaussian mixtures drawn on the device), stored as FP8
    E4M3 with per-dimension scales, exact top-100 L2 through pdx_server (CUDA
    graphs per (collection, batch bucket), autotuned launch shapes). The query
    stream is 1000 batches of log-uniform size 1..4096, each to one collection;
    a step is a tenth of the stream. The line adds queries/s per batch-size
    bucket and the same stream on FP32 storage."""
    import numpy as np
    import torch

    import pdx_synth
    from paper_2503_04422_gb300 import build as pbuild
    pbuild.build()
    from paper_2503_04422_gb300 import pdx

    torch.cuda.set_device(local_rank)
    spec = WORKLOADS[args.workload]
    k = spec["k"]
    colls = pdx_synth.serving_collections()
    if args.n:   # smaller collections (profiling / quick runs)
        colls = [pdx_synth.Collection(min(c.n, args.n), c.d, c.seed) for c in colls]
    qpool = 4096
    t0 = time.perf_counter()
    ix8, ix32, qs = [], [], []
    for c in colls:
        x, q = pdx_synth.mixture_device(c.n, c.d, qpool, c.seed)
        ix8.append(pdx.pdx_build_layout(x, storage="fp8"))
        if not args.no_f32_compare:
            ix32.append(pdx.pdx_build_layout(x))
        qs.append(q)
        del x
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    build_s = time.perf_counter() - t0
    stream_spec = pdx_synth.serving_stream(spec["batches"], len(colls), spec["max_batch"])
    K = args.steps
    per_step = (len(stream_spec) + K - 1) // K
    tune_path = os.path.join(tempfile.gettempdir(), f"pdx_tune_{os.getpid()}.json")
    st = torch.cuda.current_stream()

    def batches():
        off = [0] * len(colls)
        out = []
        for ci, b in stream_spec:
            o = off[ci] % (qpool - b + 1)
            off[ci] += b
            out.append((ci, b, qs[ci][o:o + b]))
        return out

    plan = batches()
    outs = {b: (torch.empty((b, k), dtype=torch.float32, device="cuda"),
                torch.empty((b, k), dtype=torch.int64, device="cuda")) for b in sorted({b for _, b, _ in plan})}

    def run_stream(srv, timed):
        """Runs the stream; returns (step ms list, per-batch (size, ms))."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in plan]
        step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for i, (ci, b, q) in enumerate(plan):
            if i % per_step == 0:
                step_ev[i // per_step][0].record(st)
            ev[i][0].record(st)
            srv.search(ci, q, out=outs[b])
            ev[i][1].record(st)
            if (i + 1) % per_step == 0 or i + 1 == len(plan):
                step_ev[i // per_step][1].record(st)
        torch.cuda.synchronize()
        if not timed:
            return None, None
        return ([a.elapsed_time(b_) for a, b_ in step_ev],
                [(b, ev[i][0].elapsed_time(ev[i][1])) for i, (_, b, _) in enumerate(plan)])

    def serve(indexes, cache):
        srv = pdx.Server(indexes, k=k, max_batch=spec["max_batch"], use_graphs=True, autotune=True,
                         tune_cache=cache, pruner=spec["pruner"])
        for _ in range(max(1, args.warmup // 3)):     # tunes every (collection, bucket) and captures graphs
            run_stream(srv, False)
        launches0 = pdx.pdx_kernel_launches()
        clocks = ClockSampler(local_rank)
        clocks.start()
        step_ms, per_batch = run_stream(srv, True)
        clk = clocks.stop()
        launches = pdx.pdx_kernel_launches() - launches0
        info = srv.info
        return srv, step_ms, per_batch, clk, launches, info

    srv8, step_ms, per_batch, clk, launches, info8 = serve(ix8, tune_path)
    total_q = sum(b for _, b, _ in plan)
    tot_ms = sum(step_ms)
    value = total_q / (tot_ms / 1e3)
    buckets = {}
    for b, ms in per_batch:
        key = 1 << (b - 1).bit_length()
        qn, tm = buckets.get(key, (0, 0.0))
        buckets[key] = (qn + b, tm + ms)
    per_bucket = {str(kk): round(v[0] / (v[1] / 1e3), 1) for kk, v in sorted(buckets.items())}
    srv8.free()
    f32 = None
    if ix32:
        srv32, sm32, _, _, _, _ = serve(ix32, tune_path + ".f32")
        f32 = {"value": total_q / (sum(sm32) / 1e3), "unit": "queries/s"}
        srv32.free()
    # end to end: the same stream with host query and output buffers
    e2e = None
    if not args.no_e2e:
        srv = pdx.Server(ix8, k=k, max_batch=spec["max_batch"], use_graphs=True, autotune=True, tune_cache=tune_path,
                         pruner=spec["pruner"])
        hq = [(ci, b, q.cpu().pin_memory()) for ci, b, q in plan]
        hout = {b: (torch.empty((b, k), dtype=torch.float32).pin_memory(),
                    torch.empty((b, k), dtype=torch.int64).pin_memory()) for b in outs}
        # warm-up: every (collection, batch bucket) of the stream gets its plan
        # and graph before the timed pass, as in the device-timed runs
        for ci, b, q in hq:
            srv.search(ci, q, out=hout[b])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ci, b, q in hq:
            srv.search(ci, q, out=hout[b])
        el = time.perf_counter() - t0
        srv.free()
        e2e = {"value": total_q / el, "unit": "queries/s",
               "h2d_bytes_per_step": int(sum(b * colls[ci].d * 4 for ci, b, _ in plan) / K),
               "d2h_bytes_per_step": int(total_q * k * 12 / K),
               "timer": "host wall clock around the calls (each call returns after its results are on the host)"}
    cpu = None
    if not args.no_cpu_baseline:
        ci = int(np.argsort([c.n for c in colls])[len(colls) // 2])
        c = colls[ci]
        x, q = pdx_synth.mixture_device(c.n, c.d, 64, c.seed)
        rate, thr, done = cpu_oracle_rate(x.cpu().numpy(), q.cpu().numpy(), k, budget_s=args.cpu_budget)
        cpu = {"value": rate, "unit": "queries/s", "cores": thr, "kind": "oracle",
               "sample": f"{done} queries against collection {ci} (n={c.n}, d={c.d}, the median size), FP64 brute force"}
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": 1, "steps": K, "warmup": args.warmup,
            "ms_per_step": tot_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp8_e4m3 (FP32 accumulate, FP32 rerank)", "data": "synthetic",
            "config": {"workload": args.workload, "collections": len(colls), "vectors": int(sum(c.n for c in colls)),
                       "values": int(sum(c.n * c.d for c in colls)), "k": k, "batches": len(plan),
                       "queries": total_q, "max_batch": spec["max_batch"], "pruner": spec["pruner"],
                       "graphs": True, "autotune": True,
                       "l2": "collections 12 GB (FP8) > L2; no flush between batches (a serving stream)"},
            "per_batch_bucket_qps": per_bucket, "fp32_storage": f32,
            "server": {"graph_launches": int(info8["graph_launches"]), "direct_launches": int(info8["direct_launches"]),
                       "tunings": int(info8["tunings"]), "workspace_bytes": int(info8["workspace_bytes"])},
            "build_s": build_s, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    try:
        os.unlink(tune_path)
        os.unlink(tune_path + ".f32")
    except OSError:
        pass


def run_serving_batch1(args, rank, world, local_rank):
    """Batch-1 latency through the serving runtime: the largest, the median and
    the smallest of the 64 serving collections (FP8, exact top-100), one query
    per call, graphs and the tuner on. Each collection takes --warmup calls
    (tuning and graph capture happen there), then --steps timed calls, each
    bracketed by CUDA events; the line gives the median device time per call
    and queries/s at that median for the median collection."""
    import numpy as np
    import torch

    import pdx_synth
    from paper_2503_04422_gb300 import build as pbuild
    pbuild.build()
    from paper_2503_04422_gb300 import pdx

    torch.cuda.set_device(local_rank)
    spec = WORKLOADS[args.workload]
    k = spec["k"]
    colls = pdx_synth.serving_collections()
    order = np.argsort([c.n for c in colls])
    picks = {"largest": int(order[-1]), "median": int(order[len(order) // 2]), "smallest": int(order[0])}
    if args.b1_collection != "all":
        picks = {args.b1_collection: picks[args.b1_collection]}
    nq = args.steps + args.warmup
    ixs, qs = [], []
    for ci in picks.values():
        c = colls[ci]
        x, q = pdx_synth.mixture_device(c.n, c.d, nq, c.seed)
        ixs.append(pdx.pdx_build_layout(x, storage=spec["storage"]))
        qs.append(q)
        del x
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    srv = pdx.Server(ixs, k=k, max_batch=4096, use_graphs=True, autotune=True, pruner=spec["pruner"])
    out = (torch.empty((1, k), dtype=torch.float32, device="cuda"), torch.empty((1, k), dtype=torch.int64, device="cuda"))
    st = torch.cuda.current_stream()
    res = {}
    launches = 0
    clocks = ClockSampler(local_rank)
    clocks.start()
    for j, (name, ci) in enumerate(picks.items()):
        for r in range(args.warmup):
            srv.search(j, qs[j][r:r + 1], out=out)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        l0 = pdx.pdx_kernel_launches()
        for r in range(args.steps):
            ev[r][0].record(st)
            srv.search(j, qs[j][args.warmup + r:args.warmup + r + 1], out=out)
            ev[r][1].record(st)
        torch.cuda.synchronize()
        launches += pdx.pdx_kernel_launches() - l0
        ms = sorted(a.elapsed_time(b) for a, b in ev)
        c = colls[ci]
        res[name] = {"collection": f"{c.n} x {c.d}", "median_ms": ms[len(ms) // 2], "min_ms": ms[0], "max_ms": ms[-1]}
    clk = clocks.stop()
    srv.free()
    main = res.get("median") or next(iter(res.values()))
    line = {"metric": METRIC, "value": 1e3 / main["median_ms"], "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["median_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp8_e4m3 (FP32 accumulate, FP32 rerank)", "data": "synthetic",
            "config": {"workload": args.workload, "k": k, "batch": 1, "collections": res, "graphs": True,
                       "autotune": True, "timer": "CUDA events around each call (median over the timed calls)"},
            "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)


def run_layouts(args, rank, world, local_rank):
    """The layout comparison (Sec. 3 Fig. 3, Table 3's kernel study, N-ary +
    gather and DSM in Sec. 7) on one workload: exact top-k by a linear scan
    (no pruning) over PDX blocks, N-ary rows, N-ary rows transposed on the fly
    through shared memory, and the fully dimension-major DSM copy, all with
    the same lean kernel shape (layout scans), plus the library's PDX scan.
    Every layout must return the same ids. The line reports each layout's
    queries/s and logical GB/s (n * d * 4 bytes per query) and the PDX
    speedup over N-ary, the paper's Table 3 ratio."""
    import numpy as np
    import torch

    import pdx_synth
    from paper_2503_04422_gb300 import build as pbuild
    pbuild.build()
    from paper_2503_04422_gb300 import pdx

    torch.cuda.set_device(local_rank)
    base = args.layout_workload
    k = WORKLOADS[base]["k"]
    nq = args.nq or pdx_synth.WORKLOADS[base]["nq"]
    x, q = pdx_synth.make(base, n=args.n, nq=nq)
    n, d = x.shape
    ix = pdx.pdx_build_layout(torch.from_numpy(x).cuda(), keep_dsm=True)
    torch.cuda.synchronize()
    qd = torch.from_numpy(q).cuda()
    od = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    oi = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    peak, peak_kind = _peak_hbm()
    res, ref = {}, None
    for layout in ("pdx", "pdx_kernel", "nary", "nary_gather", "dsm"):
        opts = pdx.search_opts(pruner="none", engine="scan", layout=layout)
        for _ in range(args.warmup):
            pdx.pdx_search_exact(ix, qd, k, opts=opts, out=(od, oi))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record()
            pdx.pdx_search_exact(ix, qd, k, opts=opts, out=(od, oi))
            ev[i][1].record()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        ids = oi.cpu().numpy()
        if ref is None:
            ref = ids
        gbs = nq * n * d * 4.0 / (ms / 1e3) / 1e9
        res[layout] = {"qps": nq / (ms / 1e3), "ms": ms, "logical_gbs": gbs, "frac_of_hbm": gbs / peak,
                       "same_ids": bool(np.array_equal(ids, ref))}
        print(json.dumps({"layout": layout, **res[layout]}), file=sys.stderr, flush=True)
    best = res["pdx_kernel"]
    line = {"metric": METRIC, "value": best["qps"], "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"layouts_{base}", "n": n, "d": d, "nq": nq, "k": k, "pruner": "none",
                       "l2": "256 MB L2 flush between timed steps (untimed)"},
            "layouts": res,
            "pdx_over_nary": res["pdx_kernel"]["qps"] / res["nary"]["qps"],
            "pdx_over_gather": res["pdx_kernel"]["qps"] / res["nary_gather"]["qps"],
            "pdx_over_dsm": res["pdx_kernel"]["qps"] / res["dsm"]["qps"],
            "peak": peak, "peak_kind": peak_kind}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bond_exact_1m_d768", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="smaller collection (profiling); default = workload size")
    ap.add_argument("--nq", type=int, default=None, help="queries per GPU; default = workload size")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "fp8"])
    ap.add_argument("--pruner", default=None, choices=["none", "bond", "cs_ip"],
                    help="exact workloads: override the workload's pruner")
    ap.add_argument("--engine", default=None, choices=["auto", "scan", "tensor"],
                    help="unpruned exact search: PDX scan or tensor-core GEMM (default tensor)")
    ap.add_argument("--pruners", default="ads,bsa,bond", help="IVF workload: pruners to sweep")
    ap.add_argument("--recall-queries", type=int, default=256,
                    help="IVF workload: queries whose recall is checked against the FP64 oracle")
    ap.add_argument("--traces", type=int, default=None, help="learned-order workload: training queries")
    ap.add_argument("--epochs", type=int, default=30, help="learned-order workload: training epochs")
    ap.add_argument("--no-f32-compare", action="store_true", help="serving workload: skip the FP32-storage stream")
    ap.add_argument("--b1-collection", default="all", choices=["all", "largest", "median", "smallest"],
                    help="batch-1 serving workload: which collections")
    ap.add_argument("--first-step", type=int, default=None, help="exact and IVF workloads: first fetch step (default 4)")
    ap.add_argument("--no-alt", action="store_true", help="exact workload: skip the tensor-engine companion line")
    ap.add_argument("--ctas-per-sm", type=int, default=None, help="exact and IVF workloads: resident scan CTAs per SM")
    ap.add_argument("--start-vectors", type=int, default=None, help="exact workloads: START scan size (default 1024)")
    ap.add_argument("--selection-threshold", type=float, default=None,
                    help="exact workloads: survivor share below which a block enters PRUNE (default 0.2)")
    ap.add_argument("--shard", action="store_true",
                    help="exact workload: split the collection over the ranks by id range (strong scaling)")
    ap.add_argument("--layout-workload", default="plain_scan_10k_d128",
                    choices=["plain_scan_10k_d128", "bond_exact_1m_d768"],
                    help="layouts workload: the collection the layouts are compared on")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload.startswith("ivf"):
        run_ivf(args, rank, world, local_rank)
    elif args.workload.startswith("learned"):
        run_learned(args, rank, world, local_rank)
    elif args.workload == "serving_batch1_fp8":
        run_serving_batch1(args, rank, world, local_rank)
    elif args.workload.startswith("serving"):
        run_serving(args, rank, world, local_rank)
    elif args.workload == "layouts":
        run_layouts(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
