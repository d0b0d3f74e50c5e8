"""Seeded synthetic workloads for fixed-radius search (inputs only).

This module draws points, query sets and radii.  It holds none of the
search method's arithmetic, so both the CPU oracle and the CUDA path take
their inputs from here and from nowhere else.

Every generator uses numpy's ``Generator(PCG64(seed))`` and returns FP32
row-major points; radii are float64 and are passed unchanged to every path.

Workloads (all synthetic; the paper's real-world sets of Section 6.3 are not
used):

* ``gmm_iso``       -- isotropic Gaussian mixture (n=2,000, d=8, 5 clusters);
* ``gmm_aniso``     -- 50-cluster anisotropic, rotated mixture (n=1e6, d=16);
* ``lowrank_img``   -- 784-dim images near a rank-20 subspace (n=70,000);
* ``ragged_batch``  -- 256 independent mixtures of uneven n and d;
* ``blobs3d``       -- 3-d particle blobs plus uniform noise (n=5e5, DBSCAN);
* ``uniform_cube``  -- uniform points in [0,1]^d (the Section 6.1/6.2 data);
* ``glove_like``    -- word-vector-like directions for cosine / angular search
                       (a synthetic stand-in for the GloVe100 vectors of
                       Section 6.3; R holds a cosine-distance bound);
* ``mips_like``     -- the same vectors with separate queries for the
                       inner-product threshold search (R holds the threshold).

The radius for a workload is a quantile of the pairwise Euclidean distances
of a seeded subsample (all i<j pairs, ``numpy.quantile`` default linear
method); the quantile is chosen so that a point has about ``k`` neighbours on
average, i.e. ``k/(n-1)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.distance import pdist

SEED_BASE = 2212076790


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Workload:
    """One fixed-radius search problem: points P (n x d, FP32), queries Q
    (m x d, FP32, or None for a self-join), radius R (float64)."""
    name: str
    P: np.ndarray
    Q: np.ndarray | None
    R: float
    query_ids: np.ndarray | None = None   # rows of P used as queries, if any
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.P.shape[0])

    @property
    def d(self) -> int:
        return int(self.P.shape[1])

    @property
    def m(self) -> int:
        return self.n if self.Q is None else int(self.Q.shape[0])


def subsample_radius(P: np.ndarray, q: float, sub: int, rng: np.random.Generator) -> float:
    """Quantile ``q`` of the i<j pairwise distances of a seeded subsample of
    ``min(sub, n)`` rows of P (distances in float64)."""
    n = P.shape[0]
    k = min(sub, n)
    idx = np.sort(rng.choice(n, size=k, replace=False))
    dist = pdist(P[idx].astype(np.float64))
    return float(np.quantile(dist, q))


def _mixture(rng, n, centres, std_axes, rot=None):
    k, d = centres.shape
    lab = rng.integers(0, k, size=n)
    z = rng.standard_normal((n, d)) * std_axes[None, :]
    if rot is not None:
        z = z @ rot.T
    return (centres[lab] + z).astype(np.float32), lab


def gmm_iso(n: int = 2000, d: int = 8, clusters: int = 5, m: int = 500,
            quantile: float = 0.005, sub: int = 1000, seed: int = SEED_BASE + 1) -> Workload:
    """Isotropic mixture: centres U[-10,10]^d, std 1.0; m queries drawn from
    the data without replacement; R = 0.5% quantile over 1,000 points."""
    rng = rng_for(seed)
    centres = rng.uniform(-10.0, 10.0, size=(clusters, d))
    P, lab = _mixture(rng, n, centres, np.ones(d))
    qid = rng.choice(n, size=min(m, n), replace=False)
    R = subsample_radius(P, quantile, sub, rng)
    return Workload("gmm_iso", P, P[qid].copy(), R, query_ids=qid, extra={"labels": lab})


def random_rotation(rng, d):
    a = rng.standard_normal((d, d))
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))[None, :]


def gmm_aniso(n: int = 1_000_000, d: int = 16, clusters: int = 50, nbrs: float = 50.0,
              sub: int = 4000, seed: int = SEED_BASE + 2, queries: int = 0) -> Workload:
    """Anisotropic rotated mixture: per-axis std 0.9^i, one random rotation,
    centres U[-20,20]^d; self-join; R gives ~``nbrs`` neighbours per point.
    With ``queries`` > 0, that many further draws of the same mixture form a
    separate query set (the points and R are those of the self-join)."""
    rng = rng_for(seed)
    centres = rng.uniform(-20.0, 20.0, size=(clusters, d))
    rot = random_rotation(rng, d)
    std = 0.9 ** np.arange(d)
    P, lab = _mixture(rng, n, centres, std, rot)
    R = subsample_radius(P, nbrs / (n - 1), sub, rng)
    if queries > 0:
        Q, _ = _mixture(rng, queries, centres, std, rot)
        return Workload("gmm_aniso_oos", P, Q, R, extra={"labels": lab})
    return Workload("gmm_aniso", P, None, R, extra={"labels": lab})


def lowrank_img(n: int = 70_000, d: int = 784, rank: int = 20, clusters: int = 10,
                noise: float = 0.05, nbrs: float = 30.0, sub: int = 4000,
                seed: int = SEED_BASE + 3) -> Workload:
    """Image-like data: 10 centres 0.5 + B z (B orthonormal d x rank,
    z ~ N(0, 1.25^2 I)), plus N(0, noise^2) per coordinate, clipped to [0,1];
    self-join; R gives ~``nbrs`` neighbours per point."""
    rng = rng_for(seed)
    B, _ = np.linalg.qr(rng.standard_normal((d, rank)))
    z = rng.standard_normal((clusters, rank)) * 1.25
    centres = 0.5 + z @ B.T
    lab = rng.integers(0, clusters, size=n)
    X = np.empty((n, d), dtype=np.float32)
    step = 8192
    for s in range(0, n, step):
        e = min(n, s + step)
        blk = centres[lab[s:e]] + noise * rng.standard_normal((e - s, d))
        X[s:e] = np.clip(blk, 0.0, 1.0)
    R = subsample_radius(X, nbrs / (n - 1), sub, rng)
    return Workload("lowrank_img", X, None, R, extra={"labels": lab})


def blobs3d(n: int = 500_000, blobs: int = 200, noise_frac: float = 0.10, box: float = 100.0,
            std: float = 0.5, eps: float = 0.4, min_pts: int = 10,
            seed: int = SEED_BASE + 5) -> Workload:
    """Particle-like 3-d data: (1-noise_frac) n points from ``blobs``
    isotropic blobs (centres U[0,box]^3, std 0.5) plus noise_frac n uniform
    points in [0,box]^3; DBSCAN with eps, minPts; rows are shuffled."""
    rng = rng_for(seed)
    n_noise = int(round(noise_frac * n))
    n_blob = n - n_noise
    centres = rng.uniform(0.0, box, size=(blobs, 3))
    lab = rng.integers(0, blobs, size=n_blob)
    pb = centres[lab] + std * rng.standard_normal((n_blob, 3))
    pn = rng.uniform(0.0, box, size=(n_noise, 3))
    P = np.concatenate([pb, pn]).astype(np.float32)
    perm = rng.permutation(n)
    return Workload("blobs3d", P[perm].copy(), None, float(eps),
                    extra={"min_pts": int(min_pts)})


def ragged_batch(sets: int = 256, n_lo: int = 1000, n_hi: int = 200_000,
                 dims=(2, 3, 8, 32), k_lo: int = 3, k_hi: int = 20, qfrac: float = 0.10,
                 nbrs: float = 20.0, sub: int = 4000, seed: int = SEED_BASE + 4,
                 n_scale: float = 1.0) -> list[Workload]:
    """256 independent mixtures: n log-uniform in [n_lo, n_hi] (times
    ``n_scale``), d from ``dims``, 3-20 clusters (centres U[-10,10]^d, std 1),
    10% of rows as queries, per-set R for ~``nbrs`` neighbours."""
    rng = rng_for(seed)
    out = []
    for s in range(sets):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))) * n_scale))
        n = max(n, 2)
        d = int(rng.choice(np.asarray(dims)))
        k = int(rng.integers(k_lo, k_hi + 1))
        centres = rng.uniform(-10.0, 10.0, size=(k, d))
        P, _ = _mixture(rng, n, centres, np.ones(d))
        m = max(1, int(round(qfrac * n)))
        qid = rng.choice(n, size=m, replace=False)
        R = subsample_radius(P, min(1.0, nbrs / (n - 1)), sub, rng)
        out.append(Workload(f"ragged_{s}", P, P[qid].copy(), R, query_ids=qid))
    return out


def uniform_cube(n: int, d: int, seed: int) -> np.ndarray:
    """n points uniform in [0,1]^d (Sections 6.1 and 6.2), FP32."""
    return rng_for(seed).uniform(0.0, 1.0, size=(n, d)).astype(np.float32)


def gaussian_blob(n: int, d: int, s: float, seed: int) -> np.ndarray:
    """Elongated Gaussian blob of Section 5: std [1, s, ..., s], FP32."""
    std = np.full(d, s)
    std[0] = 1.0
    return (rng_for(seed).standard_normal((n, d)) * std[None, :]).astype(np.float32)


def glove_like(n: int = 200_000, d: int = 100, clusters: int = 200, spread: float = 0.75,
               nbrs: float = 20.0, sub: int = 4000, seed: int = SEED_BASE + 6) -> Workload:
    """Direction data for cosine / angular search: cluster directions
    N(0, I_d), members = direction + spread * N(0, I_d), each row scaled by a
    log-normal magnitude (exp N(0, 0.5^2); the cosine ignores it); self-join.
    R is a cosine-distance bound: the nbrs/(n-1) quantile of the i<j cosine
    distances of a seeded subsample (scipy pdist, metric "cosine")."""
    rng = rng_for(seed)
    dirs = rng.standard_normal((clusters, d))
    lab = rng.integers(0, clusters, size=n)
    X = np.empty((n, d), dtype=np.float32)
    step = 65536
    for s0 in range(0, n, step):
        e = min(n, s0 + step)
        blk = dirs[lab[s0:e]] + spread * rng.standard_normal((e - s0, d))
        X[s0:e] = blk * np.exp(0.5 * rng.standard_normal((e - s0, 1)))
    k = min(sub, n)
    idx = np.sort(rng.choice(n, size=k, replace=False))
    c = float(np.quantile(pdist(X[idx].astype(np.float64), metric="cosine"), nbrs / (n - 1)))
    return Workload("glove_like", X, None, c, extra={"labels": lab, "measure": "cosine distance"})


def mips_like(n: int = 200_000, d: int = 100, m: int = 10_000, clusters: int = 200,
              spread: float = 0.75, nbrs: float = 20.0, sub: int = 4000,
              seed: int = SEED_BASE + 7) -> Workload:
    """Inner-product threshold search on word-vector-like rows (the vectors of
    ``glove_like``, magnitudes kept) with m queries drawn the same way; R is
    the threshold tau: the 1 - nbrs/n quantile of the dot products of a
    seeded subsample of points with a subsample of queries (float64)."""
    rng = rng_for(seed)
    dirs = rng.standard_normal((clusters, d))

    def draw(k):
        lab = rng.integers(0, clusters, size=k)
        X = dirs[lab] + spread * rng.standard_normal((k, d))
        return (X * np.exp(0.5 * rng.standard_normal((k, 1)))).astype(np.float32)
    P = draw(n)
    Q = draw(m)
    ps = P[rng.choice(n, size=min(sub, n), replace=False)].astype(np.float64)
    qs = Q[rng.choice(m, size=min(sub // 4, m), replace=False)].astype(np.float64)
    tau = float(np.quantile(ps @ qs.T, 1.0 - nbrs / n))
    return Workload("mips_like", P, Q, tau, extra={"measure": "inner product"})


def by_name(name: str, **kw):
    """Workload factory by name (sizes overridable for smaller parity cases)."""
    table = {"gmm_iso": gmm_iso, "gmm_aniso": gmm_aniso, "lowrank_img": lowrank_img,
             "blobs3d": blobs3d, "ragged_batch": ragged_batch, "glove_like": glove_like,
             "mips_like": mips_like}
    return table[name](**kw)
