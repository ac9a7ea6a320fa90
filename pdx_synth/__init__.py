"""Seeded synthetic inputs shaped like the PDX paper's workloads.

This module only draws random numbers: it holds none of the search method's
arithmetic, so both the CPU oracle (``oracle/``) and the CUDA path
(``paper_2503_04422_gb300``) may consume its output without sharing any code
with each other.

The paper evaluates on real embedding collections (Table 1: GloVe, SIFT,
Contriever, arXiv, GIST, OpenAI, ...). Those files are not available here, so
every generator below is a synthetic stand-in with the dimensionality, size and
value structure (normal vs. skewed per-dimension spread, clustering, unit norm)
of the collection it replaces. Recipes:

* ``iid_normal``           i.i.d. N(0,1) vectors, as used for the kernel study
                           (Sec. 6.2: "standardly distributed randomly generated
                           float32").
* ``gaussian_mixture``     256 centres c ~ N(0, I); vector = centre + sigma*z with
                           per-dimension spread sigma_j = pi(j)^-1/2 under a seeded
                           permutation pi (skewed dimensions, like GIST/Contriever);
                           queries are drawn the same way around random centres.
                           ``rotate=True`` multiplies everything by a seeded random
                           orthogonal matrix (the generator's own rotation, not the
                           one ADSampling later applies).
* ``embedding_like``       unit-norm vectors around 4096 unit centres with a rank-64
                           anisotropic term of norm ~0.3 plus isotropic noise of norm
                           0.05 (stand-in for OpenAI/1536 text embeddings).
* ``serving_collections``  64 collections with log-uniform sizes and D drawn from
                           {96, 384, 1024}, each a Gaussian mixture (drawn on the
                           device by ``mixture_device`` at full size).

Seeds: base seed 2503 plus the workload index, PCG64 streams keyed by
``[seed, stream, chunk]`` so that any chunk can be regenerated on its own.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 2503
_CHUNK = 1 << 16


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(list(key)))


def iid_normal(n: int, d: int, nq: int, seed: int = BASE_SEED):
    """Base vectors and queries with i.i.d. N(0,1) float32 entries."""
    x = _rng(seed, 0).standard_normal((n, d), dtype=np.float32)
    q = _rng(seed, 1).standard_normal((nq, d), dtype=np.float32)
    return x, q


def random_orthogonal(d: int, seed: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the
    signs of R's diagonal folded into Q (Mezzadri's recipe). Returned as
    float32, row-major [d][d]."""
    g = _rng(seed, 7).standard_normal((d, d))
    qm, r = np.linalg.qr(g)
    qm = qm * np.sign(np.diag(r))[None, :]
    return qm.astype(np.float32)


def anisotropic_gaussian(n: int, d: int, nq: int, decay: float = 0.9, seed: int = BASE_SEED + 8):
    """Vectors and queries from one zero-mean Gaussian whose covariance has
    the eigenvalues decay^(2j) (well separated) along the axes of a seeded
    random orthogonal basis: a workload whose principal components are
    distinct and not aligned with the storage axes."""
    sig = (decay ** np.arange(d)).astype(np.float64)
    basis = random_orthogonal(d, seed + 1).astype(np.float64)
    x = ((_rng(seed, 0).standard_normal((n, d)) * sig) @ basis.T).astype(np.float32)
    q = ((_rng(seed, 1).standard_normal((nq, d)) * sig) @ basis.T).astype(np.float32)
    return x, q


def mips_vectors(n: int, d: int, nq: int, decay: float = 0.93, norm_spread: float = 1.0,
                 seed: int = BASE_SEED + 9):
    """Inner-product workload with varied norms: coordinates independent,
    zero-mean Gaussian with standard deviation decay^j in storage order (the
    energy sits in the leading coordinates, as after a PCA projection), and
    each vector scaled by exp(u), u uniform in [-norm_spread, norm_spread].
    Queries follow the same coordinates without the norm scaling."""
    sig = (decay ** np.arange(d)).astype(np.float64)
    scale = np.exp(_rng(seed, 2).uniform(-norm_spread, norm_spread, size=(n, 1)))
    x = (_rng(seed, 0).standard_normal((n, d)) * sig * scale).astype(np.float32)
    q = (_rng(seed, 1).standard_normal((nq, d)) * sig).astype(np.float32)
    return x, q


@dataclass
class MixtureSpec:
    n: int
    d: int
    nq: int
    n_centres: int = 256
    seed: int = BASE_SEED + 1
    rotate: bool = False


def _mixture_params(spec: MixtureSpec):
    rng = _rng(spec.seed, 100)
    centres = rng.standard_normal((spec.n_centres, spec.d)).astype(np.float32)
    perm = rng.permutation(spec.d)
    sigma = (np.arange(1, spec.d + 1, dtype=np.float64) ** -0.5)[perm].astype(np.float32)
    rot = random_orthogonal(spec.d, spec.seed + 1000) if spec.rotate else None
    return centres, sigma, rot


def _mixture_rows(spec: MixtureSpec, centres, sigma, rot, count: int, stream: int,
                  out: np.ndarray | None = None) -> np.ndarray:
    if out is None:
        out = np.empty((count, spec.d), dtype=np.float32)
    for c0 in range(0, count, _CHUNK):
        c1 = min(count, c0 + _CHUNK)
        rng = _rng(spec.seed, stream, c0 // _CHUNK)
        lab = rng.integers(0, spec.n_centres, size=c1 - c0)
        z = rng.standard_normal((c1 - c0, spec.d), dtype=np.float32)
        blk = centres[lab] + sigma[None, :] * z
        if rot is not None:
            blk = blk @ rot.T
        out[c0:c1] = blk
    return out


def gaussian_mixture(spec: MixtureSpec):
    """Returns (x [n][d], q [nq][d]) float32."""
    centres, sigma, rot = _mixture_params(spec)
    x = _mixture_rows(spec, centres, sigma, rot, spec.n, 1)
    q = _mixture_rows(spec, centres, sigma, rot, spec.nq, 2)
    return x, q


def embedding_like(n: int, d: int, nq: int, n_clusters: int = 4096, rank: int = 64,
                   seed: int = BASE_SEED + 3):
    """Unit-norm vectors: x = mu_c + U_c z * (0.3/8) + eps * (0.05/sqrt(d)),
    U_c in R^{d x rank} with N(0, 1/d) entries (so the anisotropic term has
    norm ~0.3), eps ~ N(0, I) (noise of norm ~0.05), then x /= ||x||.
    mu_c are unit vectors. U_c is regenerated from its own stream per cluster
    so the generator never holds all 4096 of them."""
    rng = _rng(seed, 200)
    mu = rng.standard_normal((n_clusters, d)).astype(np.float32)
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)

    def rows(count: int, stream: int) -> np.ndarray:
        out = np.empty((count, d), dtype=np.float32)
        lab = _rng(seed, stream, 999_999).integers(0, n_clusters, size=count)
        order = np.argsort(lab, kind="stable")
        bounds = np.searchsorted(lab[order], np.arange(n_clusters + 1))
        for c in range(n_clusters):
            idx = order[bounds[c]:bounds[c + 1]]
            if idx.size == 0:
                continue
            u = _rng(seed, 300, c).standard_normal((d, rank)).astype(np.float32) / np.float32(math.sqrt(d))
            r2 = _rng(seed, stream, c)
            z = r2.standard_normal((idx.size, rank), dtype=np.float32)
            eps = r2.standard_normal((idx.size, d), dtype=np.float32)
            v = mu[c][None, :] + (z @ u.T) * np.float32(0.3 / 8.0) + eps * np.float32(0.05 / math.sqrt(d))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            out[idx] = v
        return out

    return rows(n, 1), rows(nq, 2)


def hetero_mixture(n: int, d: int, nq: int, n_centres: int = 64, seed: int = BASE_SEED + 6):
    """Gaussian mixture whose per-dimension spread varies strongly across
    dimensions (log-uniform in [0.05, 2]) around centres ~ N(0, 0.25 I): the
    distance-to-means order alone does not see the spread, so a learned
    correction has something to learn."""
    rng = _rng(seed, 600)
    sig = np.exp(rng.uniform(math.log(0.05), math.log(2.0), d)).astype(np.float32)
    cen = (rng.standard_normal((n_centres, d)) * 0.5).astype(np.float32)

    def rows(count, stream):
        r = _rng(seed, stream)
        lab = r.integers(0, n_centres, count)
        return (cen[lab] + sig * r.standard_normal((count, d), dtype=np.float32)).astype(np.float32)

    return rows(n, 1), rows(nq, 2)


@dataclass
class Collection:
    n: int
    d: int
    seed: int


def serving_collections(n_coll: int = 64, n_min: int = 10_000, n_max: int = 2_000_000,
                        dims=(96, 384, 1024), seed: int = BASE_SEED + 4):
    """Specs of the uneven serving workload: sizes log-uniform in
    [n_min, n_max], D uniform over ``dims``."""
    rng = _rng(seed, 400)
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_coll)).astype(np.int64)
    ds = rng.choice(np.asarray(dims), size=n_coll)
    return [Collection(int(ns[i]), int(ds[i]), seed * 1000 + i) for i in range(n_coll)]


def collection_data(c: Collection, nq: int = 0):
    return gaussian_mixture(MixtureSpec(n=c.n, d=c.d, nq=nq, seed=c.seed))


def mixture_device(n: int, d: int, nq: int, seed: int, n_centres: int = 256, device="cuda"):
    """The ``gaussian_mixture`` recipe (centres ~ N(0, I), spread
    sigma_j = pi(j)^-1/2 under a seeded permutation) drawn with torch's
    generator on ``device``, for collections too large to draw on the host.
    Deterministic for a given seed and device type; returns (x, q) tensors."""
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    centres = torch.randn(n_centres, d, generator=g, device=device)
    perm = torch.randperm(d, generator=g, device=device)
    sigma = (torch.arange(1, d + 1, device=device, dtype=torch.float64) ** -0.5)[perm].float()

    def rows(count):
        lab = torch.randint(0, n_centres, (count,), generator=g, device=device)
        out = torch.randn(count, d, generator=g, device=device)
        out.mul_(sigma).add_(centres[lab])
        return out

    return rows(n), rows(nq)


def serving_stream(n_batches: int, n_coll: int, max_batch: int = 4096, seed: int = BASE_SEED + 5):
    """(collection index, batch size) per batch: sizes log-uniform in [1, max_batch]."""
    rng = _rng(seed, 500)
    sizes = np.exp(rng.uniform(0.0, math.log(max_batch), size=n_batches)).astype(np.int64)
    sizes = np.clip(sizes, 1, max_batch)
    coll = rng.integers(0, n_coll, size=n_batches)
    return list(zip(coll.tolist(), sizes.tolist()))


# Named workloads (sizes as the paper-shaped configurations state them).
WORKLOADS = {
    "plain_scan_10k_d128": dict(kind="iid", n=10_000, d=128, nq=100, k=10),
    "bond_exact_1m_d768": dict(kind="mixture", n=1_000_000, d=768, nq=1_000, k=10),
    "ivf_1m_d960": dict(kind="mixture_rot", n=1_000_000, d=960, nq=10_000, k=10, nlist=1024),
    "learned_order_2m_d1536": dict(kind="embedding", n=2_000_000, d=1536, nq=5_000, k=10),
    "mips_1m_d768": dict(kind="mips", n=1_000_000, d=768, nq=1_000, k=10),
}


def make(name: str, n: int | None = None, nq: int | None = None):
    """Generate a named workload, optionally truncated to n vectors / nq queries."""
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    nq = w["nq"] if nq is None else nq
    if w["kind"] == "iid":
        return iid_normal(n, w["d"], nq, seed=BASE_SEED + 0)
    if w["kind"] == "mixture":
        return gaussian_mixture(MixtureSpec(n=n, d=w["d"], nq=nq, seed=BASE_SEED + 1))
    if w["kind"] == "mixture_rot":
        return gaussian_mixture(MixtureSpec(n=n, d=w["d"], nq=nq, seed=BASE_SEED + 2, rotate=True))
    if w["kind"] == "embedding":
        return embedding_like(n, w["d"], nq)
    if w["kind"] == "mips":
        return mips_vectors(n, w["d"], nq, decay=0.99, norm_spread=1.0)
    raise KeyError(name)
