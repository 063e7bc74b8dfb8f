"""Seeded synthetic inputs for the HNTL query path.

This module is an input generator only. It draws data vectors, queries,
attribute columns and the uniform numbers that k-means++ seeding consumes. It
holds none of the method's arithmetic (no routing, projection, PCA, scan or
selection) and imports nothing else from this package, so the CPU oracle tests
and the CUDA path can both take their inputs from it.

Clustered data (the anisotropic "manifold" stand-in of the paper's recall
table, Table 1): each cluster c has a mean m_c ~ N(0, mean_std^2 I_d), an
orthonormal basis B_c of `sub_dim` directions (QR of a d x sub_dim Gaussian),
and a point is x = m_c + B_c a + eps with a_j ~ N(0, decay^(2j)) and
eps ~ N(0, sigma^2 I_d). Values are formed in FP64 and rounded once to FP32.
Cluster sizes are equal or Zipf(s), both rounded by largest remainder.

Isotropic data (the paper's isotropic Gaussian row of Table 1): x ~ N(0, I_d).

Everything is a pure function of (shape parameters, seed, device). The small
per-cluster parameters are always drawn on the CPU, so the cluster model is the
same on every device; per-point noise is drawn on the requested device, so CPU
and CUDA draws of the points differ (each is reproducible on its own device).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch


def cluster_sizes(n: int, n_clusters: int, dist: str = "equal", zipf_s: float = 1.1) -> torch.Tensor:
    """Integer cluster sizes summing to n, by largest-remainder rounding.

    dist="equal": p_c = 1/n_clusters.  dist="zipf": p_c proportional to (c+1)^-s.
    """
    if n_clusters <= 0:
        raise ValueError("n_clusters must be positive")
    if dist == "equal":
        p = torch.full((n_clusters,), 1.0 / n_clusters, dtype=torch.float64)
    elif dist == "zipf":
        w = torch.arange(1, n_clusters + 1, dtype=torch.float64).pow(-zipf_s)
        p = w / w.sum()
    else:
        raise ValueError(f"unknown size distribution {dist!r}")
    raw = p * n
    base = torch.floor(raw).to(torch.int64)
    rem = int(n - int(base.sum()))
    frac = raw - base.to(torch.float64)
    order = torch.argsort(-frac, stable=True)
    base[order[:rem]] += 1
    return base


@dataclass
class ClusterModel:
    """Generating distribution of the clustered workloads."""

    d: int
    means: torch.Tensor  # [n_clusters, d] f64
    bases: torch.Tensor  # [n_clusters, d, sub_dim] f64, orthonormal columns
    axis_std: torch.Tensor  # [sub_dim] f64
    sigma: float
    sizes: torch.Tensor  # [n_clusters] i64

    @property
    def n_clusters(self) -> int:
        return int(self.means.shape[0])


def make_cluster_model(n: int, d: int, n_clusters: int, *, sizes: str = "equal", zipf_s: float = 1.1,
                       sub_dim: int = 8, decay: float = 0.8, sigma: float = 0.05, mean_std: float = 2.0,
                       seed: int = 0) -> ClusterModel:
    g = torch.Generator().manual_seed(int(seed))
    means = torch.randn(n_clusters, d, generator=g, dtype=torch.float64) * mean_std
    raw = torch.randn(n_clusters, d, sub_dim, generator=g, dtype=torch.float64)
    bases = torch.linalg.qr(raw).Q
    axis_std = torch.tensor([decay ** j for j in range(sub_dim)], dtype=torch.float64)
    return ClusterModel(d=d, means=means, bases=bases, axis_std=axis_std, sigma=float(sigma),
                        sizes=cluster_sizes(n, n_clusters, sizes, zipf_s))


def _draw(model: ClusterModel, labels: torch.Tensor, gen: torch.Generator, device, chunk: int) -> torch.Tensor:
    """Points x = m_c + B_c a + eps for the given cluster labels, FP64 then one rounding to FP32."""
    n = int(labels.numel())
    d = model.d
    k = int(model.axis_std.numel())
    out = torch.empty(n, d, dtype=torch.float32, device=device)
    means = model.means.to(device)
    bases = model.bases.to(device)
    axis_std = model.axis_std.to(device)
    lab_dev = labels.to(device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab = lab_dev[s:e]
        a = torch.randn(e - s, k, generator=gen, dtype=torch.float64, device=device) * axis_std
        eps = torch.randn(e - s, d, generator=gen, dtype=torch.float64, device=device) * model.sigma
        x = means[lab] + torch.bmm(bases[lab], a.unsqueeze(-1)).squeeze(-1) + eps
        out[s:e] = x.to(torch.float32)
    return out


def sample_points(model: ClusterModel, seed: int, device="cpu", chunk: int = 4096):
    """Data vectors X [N, d] f32 and their generating cluster labels [N] i64.

    Labels follow the model's cluster sizes, placed in a seeded random order.
    """
    gen = torch.Generator(device=device).manual_seed(int(seed))
    labels = torch.repeat_interleave(torch.arange(model.n_clusters), model.sizes)
    perm = torch.randperm(labels.numel(), generator=torch.Generator().manual_seed(int(seed) + 7))
    labels = labels[perm]
    return _draw(model, labels, gen, device, chunk), labels


def sample_queries(model: ClusterModel, nq: int, seed: int, device="cpu", chunk: int = 4096):
    """Queries [nq, d] f32 drawn like the data: cluster chosen with probability proportional to its size."""
    gcpu = torch.Generator().manual_seed(int(seed))
    p = model.sizes.to(torch.float64)
    labels = torch.multinomial(p / p.sum(), nq, replacement=True, generator=gcpu)
    gen = torch.Generator(device=device).manual_seed(int(seed) + 1)
    return _draw(model, labels, gen, device, chunk), labels


def isotropic(n: int, d: int, seed: int, device="cpu") -> torch.Tensor:
    """x ~ N(0, I_d), FP64 rounded once to FP32."""
    gen = torch.Generator(device=device).manual_seed(int(seed))
    return torch.randn(n, d, generator=gen, dtype=torch.float64, device=device).to(torch.float32)


def uniforms(n: int, seed: int) -> torch.Tensor:
    """n uniform numbers in [0, 1) (FP64, CPU): the draws of k-means++ seeding, passed in as inputs."""
    return torch.rand(n, generator=torch.Generator().manual_seed(int(seed)), dtype=torch.float64)


def train_subset(n: int, n_train: int, seed: int) -> torch.Tensor:
    """Sorted indices of a seeded subsample of size min(n, n_train) (k-means training set)."""
    if n_train >= n:
        return torch.arange(n, dtype=torch.int64)
    perm = torch.randperm(n, generator=torch.Generator().manual_seed(int(seed)))
    return torch.sort(perm[:n_train]).values


def attributes(n: int, seed: int, span: int = 1 << 40, device="cpu") -> torch.Tensor:
    """Per-vector int64 attribute (e.g. a timestamp), uniform in [0, span)."""
    gen = torch.Generator(device=device).manual_seed(int(seed))
    return torch.randint(0, span, (n,), generator=gen, dtype=torch.int64, device=device)


def range_filters(nq: int, seed: int, span: int = 1 << 40, selectivity: float = 0.2,
                  frac_filtered: float = 0.5) -> torch.Tensor:
    """Per-query inclusive [lo, hi] int64 ranges [nq, 2] (CPU).

    A fraction `frac_filtered` of the queries carries a range whose width is
    `selectivity` of the attribute span, placed uniformly; the rest carry the
    full int64 range (no filtering).
    """
    g = torch.Generator().manual_seed(int(seed))
    width = int(span * selectivity)
    out = torch.empty(nq, 2, dtype=torch.int64)
    out[:, 0] = torch.iinfo(torch.int64).min
    out[:, 1] = torch.iinfo(torch.int64).max
    has = torch.rand(nq, generator=g, dtype=torch.float64) < frac_filtered
    lo = torch.randint(0, span - width + 1, (nq,), generator=g, dtype=torch.int64)
    out[has, 0] = lo[has]
    out[has, 1] = lo[has] + width - 1
    return out


# Workload shapes, named by what they are (see the design notes for the recipe).
WORKLOADS = {
    "plain-10k": dict(n=10_000, d=768, n_clusters=32, sizes="equal", G=32, r=16, nq=1_000,
                      nprobe=4, C=20, k=10, seed=1001),
    "plain-1m-zipf": dict(n=1_000_000, d=768, n_clusters=1_024, sizes="zipf", G=1_024, r=32, nq=10_000,
                          batch=1_024, nprobe=16, C=100, k=10, seed=1002),
    "precision-10m": dict(n=10_000_000, d=768, n_clusters=4_096, sizes="equal", G=4_096, r=32, nq=100_000,
                          batch=16_384, nprobe=32, C=200, k=10, seed=1003, precision="bf16-fp8"),
    "precision-2.5m": dict(n=2_500_000, d=768, n_clusters=1_024, sizes="equal", G=1_024, r=32, nq=10_240,
                           batch=1_024, nprobe=32, C=200, k=10, seed=1005, precision="bf16-fp8"),
    # about four grains per cluster, capacity-bounded at 1.05 N / G rows: grains are no longer the
    # Voronoi cells of their centres, which is where a learned router has something to learn
    "router-5m": dict(n=5_000_000, d=768, n_clusters=1_024, sizes="equal", G=4_096, r=32, nq=20_000,
                      nprobe=16, C=200, k=10, seed=1004, max_grain_rows=1_282),
}


def seeds(base: int) -> dict:
    """Derived seeds of one workload: data, queries, k-means draws, router, serving arrivals."""
    return dict(data=base, queries=base + 1000, kmeans=base + 2000, router=base + 3000, serve=base + 4000)


def expected_captured_fraction(d: int, sub_dim: int, decay: float, sigma: float, r: int) -> float:
    """Closed-form share of a cluster's variance in its top-r principal directions.

    The generating covariance is B diag(decay^(2j)) B^T + sigma^2 I, with
    eigenvalues decay^(2j)+sigma^2 (j < sub_dim) and sigma^2 (d - sub_dim
    times); the top r of them over the trace.
    """
    lam = sorted([decay ** (2 * j) + sigma ** 2 for j in range(sub_dim)] + [sigma ** 2] * (d - sub_dim),
                 reverse=True)
    return sum(lam[:r]) / sum(lam)
