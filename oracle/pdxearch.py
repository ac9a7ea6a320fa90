"""The PDXearch framework run block by block, one query at a time, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

This follows the paper's description step by step; it is the reference for the
*algorithm* (which vectors are pruned when, how many dimensions are visited),
while ``oracle.knn`` is the reference for the exact *result*:

* Sec. 4 PHASE 0 START: the first block is scanned without pruning; its
  distances fill the max-heap and the k-th best becomes the threshold tau. When
  a block holds fewer than k vectors the linear scan continues into the next
  block(s) until k vectors have been seen (the paper is silent on this case).
* Sec. 4 PHASE 1 WARMUP: dimensions are fetched in steps that start at
  ``first_step`` (2) and double (2, 4, 8, ...), the last one clamped to the
  remaining dimensions. After each step the partial distances of *all*
  vectors of the block are updated and the pruning predicate is evaluated;
  a vector that fails it is discarded for good but WARMUP keeps computing
  its partial distance.
* Sec. 4 PHASE 2 PRUNE: once the fraction of not-yet-pruned vectors of the
  block is below ``selection_threshold`` (20%, Sec. 6.1) only the survivors
  (the positions array) are computed; steps keep doubling. At the last
  dimension the survivors are merged into the heap and tau tightens.
* Sec. 5 PDX-BOND: the predicate is "partial distance > tau"; dimensions are
  visited by decreasing |q_j - mu_j| where mu are the block's means
  ("distance to means"), or by decreasing q_j ("decreasing", BOND's order),
  or zone by zone: contiguous groups of ``zone_dims`` dimensions ranked by
  sum_{j in zone} (q_j - mu_j)^2, dimensions inside a zone in storage order.
  Ties in any ranking go to the lower dimension / zone index.
* Sec. 2.3 ADSampling (on data rotated by a random orthogonal matrix, dims in
  storage order): after d of D dimensions the vector is pruned when
  partial * D / d > tau * (1 + eps0 / sqrt(d))^2 -- the hypothesis test on the
  scaled partial distance with error bound eps0, written for squared distances.
* Sec. 2.3 BSA_res (on PCA-projected data, dims in storage order), pruned
  when either test fires after d visited dimensions:
  - Cauchy-Schwarz (exact): partial + (||x_r|| - ||q_r||)^2 > tau, since the
    unvisited part ||x_r - q_r||^2 is at least (||x_r|| - ||q_r||)^2;
  - error quantile: partial > tau * F(d) * (1 + m / sqrt(d))^2, where
    F(d) = sum_{visited j} lambda_j / sum_j lambda_j is the fraction of the
    collection's variance (lambda = PCA variances) in the visited dimensions,
    so partial / F(d) estimates the full distance; m -> infinity leaves only
    the exact test.

* ADSampling with PDX-BOND's query-aware order (the fusion the paper names
  as future work, Sec. 8; the reading is this build's): on rotated data the
  dimensions are visited by PDX-BOND's distance-to-means order against the
  block's means, and after d visited dimensions the vector is pruned when
  either test fires:
  - PDX-BOND (exact): partial > tau;
  - the hypothesis test, calibrated to the visited share of the expected
    distance: partial > tau * F_q(d) * (1 + eps0 / sqrt(d))^2, where
    E_j = (q_j - mu_j)^2 + var_j is the expected (q_j - x_j)^2 for a vector of
    the block (mean mu_j, population variance var_j) and F_q(d) is the sum of
    E over the visited dimensions over the sum of E over all of them. With
    storage order and equal E_j, F_q(d) = d / D and the test is ADSampling's.

* Exact inner-product pruning with the Cauchy-Schwarz bound (the exact half
  of BSA's test in Sec. 2.3, carried over to the inner product; the paper
  itself prunes only distances, and the reading is this build's): with
  ``metric="ip"`` the distance is -q.x, and after the first d dimensions in
  storage order the unvisited part q_r . x_r lies in [-||q_r|| ||x_r||,
  ||q_r|| ||x_r||]. A vector is pruned when
  partial - ||q_r|| ||x_r|| > tau, partial being the visited -sum q_j x_j and
  tau the k-th best -q.x so far: even with the most favourable unvisited part
  it cannot enter the top-k. It holds for any vector norms.

Returns the top-k plus per-query counters: values accumulated (the paper's
pruning power is 1 - visited / (n*D)), vectors pruned, and the phase at which
each block ended.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class SearchStats:
    values_visited: int = 0          # sum over vectors of dims accumulated
    vectors_seen: int = 0
    vectors_pruned: int = 0
    prune_events: list = field(default_factory=list)   # (block, vector id, dims visited at prune)


def visit_order(q, mu, order: str, zone_dims: int = 1):
    """Order in which a block's dimensions are visited (Sec. 5)."""
    d = q.shape[0]
    if order == "sequential":
        return np.arange(d)
    if order == "decreasing":
        # BOND: highest query value first; ties -> lower dim index
        return np.lexsort((np.arange(d), -q))
    if order != "dist_to_means":
        raise ValueError(order)
    score = (q - mu) ** 2
    if zone_dims <= 1:
        return np.lexsort((np.arange(d), -score))
    nz = (d + zone_dims - 1) // zone_dims
    zs = np.array([score[z * zone_dims:(z + 1) * zone_dims].sum() for z in range(nz)])
    zorder = np.lexsort((np.arange(nz), -zs))
    return np.concatenate([np.arange(z * zone_dims, min(d, (z + 1) * zone_dims)) for z in zorder])


def step_schedule(d: int, first_step: int):
    """Sizes of the fetching steps: first_step, doubling, last one clamped."""
    out, pos, s = [], 0, max(1, first_step)
    while pos < d:
        t = min(s, d - pos)
        out.append(t)
        pos += t
        s *= 2
    return out


class _Heap:
    """Best-k list ordered by (distance, id)."""

    def __init__(self, k):
        self.k = k
        self.items: list[tuple[float, int]] = []

    def merge(self, dists, ids):
        self.items.extend(zip((float(v) for v in dists), (int(i) for i in ids)))
        self.items.sort()
        del self.items[self.k:]

    @property
    def tau(self):
        return self.items[-1][0] if len(self.items) == self.k else math.inf


def pdxearch(x, q, k, blocks, pruner="bond", order="dist_to_means", zone_dims=1, first_step=2,
             selection_threshold=0.20, eps0=2.1, bsa_m=None, bsa_lambda=None, tau0=None, tau_fixed=False,
             metric="l2"):
    """One query. ``blocks`` is a list of int arrays (vector ids per PDXearch
    block, visited in list order). ``x`` is [n][D]; returns (dists, ids, stats).
    ``tau0`` optionally seeds the threshold (any k-th distance of k real
    vectors keeps the search exact); with ``tau_fixed`` the threshold stays
    tau0 instead of tightening as blocks merge into the heap. ``metric`` "ip"
    ranks by -q.x (pruners "none" and "cs_ip" only)."""
    if metric not in ("l2", "ip"):
        raise ValueError(metric)
    if (metric == "ip") != (pruner == "cs_ip") and pruner != "none":
        raise ValueError("the Cauchy-Schwarz pruner ranks inner products; the other pruners squared distances")
    x = np.asarray(x, np.float64)
    q = np.asarray(q, np.float64)
    n, d = x.shape
    heap = _Heap(k)
    st = SearchStats()
    seen = 0
    started = tau0 is not None
    tau_seed = math.inf if tau0 is None else float(tau0)
    for bi, ids in enumerate(blocks):
        ids = np.asarray(ids, np.int64)
        if ids.size == 0:
            continue
        xb = x[ids]
        if not started:
            # START: linear scan until k vectors have been seen
            full = -(xb @ q) if metric == "ip" else ((xb - q) ** 2).sum(axis=1)
            st.values_visited += ids.size * d
            st.vectors_seen += ids.size
            heap.merge(full, ids)
            seen += ids.size
            if seen >= k:
                started = True
            continue
        tau = tau_seed if tau_fixed else min(heap.tau, tau_seed)
        mass = None
        if pruner in ("bond", "none", "ads_bond"):
            mu = xb.mean(axis=0)
            dims = visit_order(q, mu, order, zone_dims)
            if pruner == "ads_bond":
                e = (q - mu) ** 2 + xb.var(axis=0)
                mass = np.concatenate([[0.0], np.cumsum(e[dims])]) / e.sum()
        else:
            dims = np.arange(d)
        partial = np.zeros(ids.size)
        pruned = np.zeros(ids.size, bool)
        positions = None          # None = WARMUP (all vectors), else PRUNE survivors
        pos = 0
        for s in step_schedule(d, first_step):
            js = dims[pos:pos + s]
            rows = np.arange(ids.size) if positions is None else positions
            if metric == "ip":
                contrib = -(xb[np.ix_(rows, js)] @ q[js])
            else:
                contrib = ((xb[np.ix_(rows, js)] - q[js]) ** 2).sum(axis=1)
            partial[rows] += contrib
            st.values_visited += rows.size * js.size
            pos += s
            if pos >= d:
                break
            test = _predicate(pruner, partial[rows], tau, pos, d, xb[rows], q, dims, pos, eps0, bsa_m, bsa_lambda,
                              None if mass is None else mass[pos])
            newly = test & ~pruned[rows]
            for r in rows[newly]:
                st.prune_events.append((bi, int(ids[r]), pos))
            pruned[rows] |= test
            alive = np.flatnonzero(~pruned)
            if alive.size == 0:
                break
            if positions is None and alive.size < selection_threshold * ids.size:
                positions = alive
            elif positions is not None:
                positions = alive
        st.vectors_seen += ids.size
        st.vectors_pruned += int(pruned.sum())
        alive = np.flatnonzero(~pruned)
        if pos >= d and alive.size:
            heap.merge(partial[alive], ids[alive])
    items = heap.items + [(math.inf, -1)] * (k - len(heap.items))
    return np.array([v for v, _ in items]), np.array([i for _, i in items], np.int64), st


def _predicate(pruner, partial, tau, dvis, d, xrows, q, dims, pos, eps0, bsa_m, bsa_lambda, mass=None):
    if pruner == "none" or not math.isfinite(tau):
        return np.zeros(partial.shape, bool)
    if pruner == "bond":
        return partial > tau
    if pruner == "ads_bond":
        return (partial > tau) | (partial > tau * mass * (1.0 + eps0 / math.sqrt(dvis)) ** 2)
    if pruner == "ads":
        return partial * (d / dvis) > tau * (1.0 + eps0 / math.sqrt(dvis)) ** 2
    if pruner == "bsa":
        rest = dims[pos:]
        rx2 = (xrows[:, rest] ** 2).sum(axis=1)
        rq2 = float((q[rest] ** 2).sum())
        cs = partial + (np.sqrt(rx2) - math.sqrt(rq2)) ** 2 > tau
        lam = np.asarray(bsa_lambda, np.float64)
        frac = float(lam[dims[:pos]].sum() / lam.sum())
        stat = partial > tau * frac * (1.0 + bsa_m / math.sqrt(dvis)) ** 2
        return cs | stat
    if pruner == "cs_ip":
        rest = dims[pos:]
        rx = np.sqrt((xrows[:, rest] ** 2).sum(axis=1))
        rq = math.sqrt(float((q[rest] ** 2).sum()))
        return partial - rq * rx > tau
    raise ValueError(pruner)


def partitions(n: int, partition_size: int):
    """Exact-search blocks (Sec. 6.6): equal horizontal partitions of at most
    ``partition_size`` vectors, in id order."""
    nparts = max(1, -(-n // partition_size))
    size = -(-n // nparts)
    return [np.arange(p * size, min(n, (p + 1) * size)) for p in range(nparts)]
