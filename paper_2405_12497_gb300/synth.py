"""Seeded synthetic workloads shaped like the paper's datasets (Table 3).

This module holds only input generation -- none of RaBitQ's arithmetic -- so
that the CUDA path, the oracle, the tests and the benchmark can all draw the
same inputs. The paper's datasets (SIFT, GIST, DEEP, ...) are not available;
the recipes below stand in for them with matching dimension, value range and
clustered structure. Data and queries use independent numpy PCG64 streams.
"""
from __future__ import annotations

from dataclasses import dataclass, replace as dataclasses_replace  # noqa: F401

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    nq: int
    n_clusters: int
    k: int
    nprobe: int
    code_bits: int = 0      # 0: smallest multiple of 64 >= d
    bq: int = 4
    eps0: float = 1.9
    kmeans_iters: int = 10
    kmeans_sample: int = 0  # 0: train k-means on every point


# The workloads of the benchmark configurations. nprobe is the default probe
# count; the benchmark sweeps it to reach recall@100 = 0.95.
TINY = Workload("tiny-gauss-10k-d128", 10_000, 128, 100, 16, 10, 4)
SIFT_LIKE = Workload("sift-like-1M-d128", 1_000_000, 128, 10_000, 4096, 100, 64)
GIST_LIKE = Workload("gist-like-1M-d960", 1_000_000, 960, 1_000, 4096, 100, 64, code_bits=1024)
DEEP_LIKE = Workload("deep-like-10M-d256", 10_000_000, 256, 10_000, 16_384, 100, 64,
                     kmeans_sample=256 * 16_384)


def gaussian_mixture(n: int, d: int, n_comp: int, sigma: float, seed: int,
                     center_seed: int = 0) -> np.ndarray:
    """Mixture of isotropic Gaussians: centers ~ N(0, I), x = center + sigma N(0, I)."""
    cen = np.random.Generator(np.random.PCG64(center_seed)).standard_normal((n_comp, d))
    g = np.random.Generator(np.random.PCG64(seed + 1000))
    comp = g.integers(0, n_comp, n)
    x = cen[comp] + sigma * g.standard_normal((n, d))
    return x.astype(np.float32)


def tiny(seed_data: int = 0, seed_query: int = 1, n: int = 10_000, d: int = 128, nq: int = 100):
    """10k x 128 mixture of 100 isotropic Gaussians (sigma 0.3), 100 queries."""
    data = gaussian_mixture(n, d, 100, 0.3, seed_data, center_seed=seed_data)
    queries = gaussian_mixture(nq, d, 100, 0.3, seed_query, center_seed=seed_data)
    return data, queries


def _chunks(n: int, step: int = 1 << 18):
    for s in range(0, n, step):
        yield s, min(n, s + step)


def sift_like(n: int, nq: int, d: int = 128, seed_data: int = 0, seed_query: int = 1,
              with_data: bool = True):
    """Non-negative integer-valued vectors in [0, 255] (SIFT-shaped): a mixture
    of n/100 components with heavy-tailed per-dimension scales s_d =
    exp(N(0, 1/4)), centers mu[c, d] = 32 s_d Exp(1), and points
    x = clip(round(mu + 24 s_d N(0, 1)), 0, 255). The overlap between
    components is set so that an IVF with K = 4096 over 1M points needs about
    64 probes for recall@100 = 0.95."""
    g = np.random.Generator(np.random.PCG64(seed_data))
    n_comp = max(10, n // 100)
    scale = np.exp(0.5 * g.standard_normal(d))
    mu = 32.0 * scale * g.exponential(1.0, (n_comp, d))

    def draw(m, seed):
        gg = np.random.Generator(np.random.PCG64(seed + 1000))
        out = np.empty((m, d), np.float32)
        for s, e in _chunks(m):
            comp = gg.integers(0, n_comp, e - s)
            x = mu[comp] + 24.0 * scale * gg.standard_normal((e - s, d))
            out[s:e] = np.clip(np.rint(x), 0, 255)
        return out

    return (draw(n, seed_data) if with_data else None), draw(nq, seed_query)


def gist_like(n: int, nq: int, d: int = 960, seed_data: int = 0, seed_query: int = 1,
              with_data: bool = True):
    """Vectors in [0, 1] from a 500-component mixture, mu ~ Beta(2, 5) per
    dimension, x = clip(mu + 0.05 N(0, 1), 0, 1) (GIST-shaped)."""
    g = np.random.Generator(np.random.PCG64(seed_data))
    mu = g.beta(2.0, 5.0, (500, d))

    def draw(m, seed):
        gg = np.random.Generator(np.random.PCG64(seed + 1000))
        out = np.empty((m, d), np.float32)
        for s, e in _chunks(m, 1 << 16):
            comp = gg.integers(0, 500, e - s)
            out[s:e] = np.clip(mu[comp] + 0.05 * gg.standard_normal((e - s, d)), 0.0, 1.0)
        return out

    return (draw(n, seed_data) if with_data else None), draw(nq, seed_query)


def deep_like(n: int, nq: int, d: int = 256, n_comp: int = 10_000, seed_data: int = 0,
              seed_query: int = 1, with_data: bool = True):
    """Unit-norm vectors from a 10k-component mixture: mu ~ N(0, I/d),
    x = normalize(mu + 0.5 N(0, I/d)) (DEEP-shaped)."""
    g = np.random.Generator(np.random.PCG64(seed_data))
    mu = g.standard_normal((n_comp, d)) / np.sqrt(d)

    def draw(m, seed):
        gg = np.random.Generator(np.random.PCG64(seed + 1000))
        out = np.empty((m, d), np.float32)
        for s, e in _chunks(m):
            comp = gg.integers(0, n_comp, e - s)
            x = mu[comp] + 0.5 * gg.standard_normal((e - s, d)) / np.sqrt(d)
            x /= np.linalg.norm(x, axis=1, keepdims=True)
            out[s:e] = x
        return out

    return (draw(n, seed_data) if with_data else None), draw(nq, seed_query)


def deep_like_device(n: int, nq: int, device, d: int = 256, n_comp: int | None = None,
                     sigma: float = 1.0, seed_data: int = 0, seed_query: int = 1,
                     with_data: bool = True):
    """DEEP-shaped unit vectors drawn directly in device memory (torch CUDA
    generator; the 10M-point set would take minutes with numpy): n_comp
    (default n/100) components mu ~ N(0, I/d), x = normalize(mu + sigma
    N(0, I/d)). With n/100 components of about 100 points each and sigma near
    1, a query's 100 nearest neighbours spread over several IVF buckets (the
    10k-component recipe puts them all in one or two). Returns torch tensors
    (data or None, queries)."""
    import math

    import torch
    n_comp = n_comp or max(10, n // 100)
    gc = torch.Generator(device=device)
    gc.manual_seed(seed_data)
    mu = torch.randn((n_comp, d), generator=gc, device=device) / math.sqrt(d)

    def draw(m, seed):
        g = torch.Generator(device=device)
        g.manual_seed(seed + 1000)
        out = torch.empty((m, d), dtype=torch.float32, device=device)
        for s in range(0, m, 1 << 20):
            e = min(m, s + (1 << 20))
            comp = torch.randint(0, n_comp, (e - s,), generator=g, device=device)
            x = mu[comp] + (sigma / math.sqrt(d)) * torch.randn((e - s, d), generator=g,
                                                                device=device)
            out[s:e] = x / x.norm(dim=1, keepdim=True)
        return out

    return (draw(n, seed_data) if with_data else None), draw(nq, seed_query)


def make(w: Workload, n: int | None = None, nq: int | None = None, seed_query: int = 1,
         with_data: bool = True):
    """Data and queries of a workload (optionally with fewer points/queries;
    another seed_query draws another query set from the same mixture, e.g.
    training queries; with_data=False skips drawing the data, returning None)."""
    n = w.n if n is None else n
    nq = w.nq if nq is None else nq
    if w is TINY or w.name.startswith("tiny"):
        return tiny(n=n, nq=nq, d=w.d, seed_query=seed_query)
    if w.name.startswith("sift"):
        return sift_like(n, nq, w.d, seed_query=seed_query, with_data=with_data)
    if w.name.startswith("gist"):
        return gist_like(n, nq, w.d, seed_query=seed_query, with_data=with_data)
    if w.name.startswith("deep"):
        return deep_like(n, nq, w.d, seed_query=seed_query, with_data=with_data)
    raise ValueError(w.name)
