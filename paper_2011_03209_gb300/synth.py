"""Seeded synthetic point clouds shaped like the mapper workloads.

This module only draws inputs: point clouds, and the DBSCAN radius picked as
a percentile of sampled pairwise distances. It holds none of the mapper
method's arithmetic (no lens, cover, clustering or nerve), so both the CUDA
path and the FP64 oracle can be fed from it without sharing code.

All draws use NumPy's PCG64 (`default_rng(seed)`), whose streams are the same
on x86-64 and AArch64, so a (workload, seed) pair names identical bytes on
every machine.

The paper's datasets (ImageNet and Cifar activation vectors, §4.3
"Datasets") are not available; the generators below stand in for them with
the same shapes: tens to a million points in 8 to 256 dimensions, clustered,
with uniform background noise.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


LENS_L2 = 0
LENS_COORD = 1
LENS_PCA = 2

PREC_FP32 = 0
PREC_BF16 = 1


@dataclasses.dataclass
class Workload:
    """One mapper problem: the point cloud plus every parameter of §3
    ("Algorithmic details in practice"): filter, n, p, eps, minPts."""

    name: str
    X: np.ndarray                 # (n, d) float32, C-contiguous
    lens_kind: tuple              # per lens dimension: LENS_*
    lens_arg: tuple               # coordinate index or principal-component index
    n_intervals: tuple
    overlap: tuple
    eps: float
    min_pts: int

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def m(self) -> int:
        return len(self.lens_kind)


def _shuffle(rng: np.random.Generator, X: np.ndarray) -> np.ndarray:
    perm = rng.permutation(X.shape[0])
    return np.ascontiguousarray(X[perm])


def eps_at_percentile(X: np.ndarray, q: float, seed: int, n_pairs: int = 100_000) -> float:
    """DBSCAN radius at the q-th percentile of sampled pairwise distances.

    Pairs (i, j), i != j, are drawn uniformly with their own seeded stream.
    The radius is placed halfway (in squared distance) between two consecutive
    sampled values, so that no sampled pair sits exactly on the boundary.
    """
    rng = np.random.default_rng([seed, 0x5E7])
    n = X.shape[0]
    i = rng.integers(0, n, size=n_pairs)
    j = rng.integers(0, n - 1, size=n_pairs)
    j = j + (j >= i)                            # uniform over j != i
    sq = np.empty(n_pairs, dtype=np.float64)
    step = 8192
    for s in range(0, n_pairs, step):
        diff = X[i[s:s + step]].astype(np.float64) - X[j[s:s + step]].astype(np.float64)
        sq[s:s + step] = np.einsum("ij,ij->i", diff, diff)
    sq.sort()
    k = max(int(math.ceil(q * n_pairs / 100.0)) - 1, 0)
    k = min(k, n_pairs - 2)
    return float(math.sqrt(0.5 * (sq[k] + sq[k + 1])))


def blobs_and_circle(seed: int = 0, n_blob: int = 1000, n_blobs: int = 4,
                     n_circle: int = 1000, d: int = 8) -> np.ndarray:
    """Isotropic Gaussian blobs (std 0.5, centres uniform in [-5, 5]^d) plus
    points on a noisy unit circle in dimensions 0-1 (noise std 0.05)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-5.0, 5.0, size=(n_blobs, d))
    parts = [c + 0.5 * rng.standard_normal((n_blob, d)) for c in centres]
    theta = rng.uniform(0.0, 2.0 * np.pi, size=n_circle)
    circ = np.zeros((n_circle, d))
    circ[:, 0] = np.cos(theta) + 0.05 * rng.standard_normal(n_circle)
    circ[:, 1] = np.sin(theta) + 0.05 * rng.standard_normal(n_circle)
    parts.append(circ)
    X = np.concatenate(parts).astype(np.float32)
    return _shuffle(rng, X)


def gaussian_mixture(n: int, d: int, k: int, seed: int, centre_box: float,
                     std_lo: float, std_hi: float, anisotropic: bool,
                     weights: np.ndarray | None = None,
                     noise_frac: float = 0.0) -> np.ndarray:
    """k Gaussian clusters (centres uniform in [-centre_box, centre_box]^d,
    std uniform in [std_lo, std_hi], per axis when `anisotropic`), optionally
    with a fraction of uniform noise in the clustered points' bounding box."""
    rng = np.random.default_rng(seed)
    n_noise = int(round(noise_frac * n))
    n_clu = n - n_noise
    if weights is None:
        weights = np.full(k, 1.0 / k)
    weights = np.asarray(weights, dtype=np.float64)
    weights = weights / weights.sum()
    sizes = np.floor(weights * n_clu).astype(np.int64)
    sizes[: n_clu - int(sizes.sum())] += 1      # hand out the remainder
    centres = rng.uniform(-centre_box, centre_box, size=(k, d)).astype(np.float32)
    if anisotropic:
        stds = rng.uniform(std_lo, std_hi, size=(k, d)).astype(np.float32)
    else:
        stds = np.repeat(rng.uniform(std_lo, std_hi, size=(k, 1)), d, axis=1).astype(np.float32)
    X = np.empty((n, d), dtype=np.float32)
    row = 0
    for c in range(k):
        z = rng.standard_normal((int(sizes[c]), d), dtype=np.float32)
        X[row:row + sizes[c]] = centres[c] + stds[c] * z
        row += int(sizes[c])
    if n_noise:
        lo = X[:n_clu].min(axis=0)
        hi = X[:n_clu].max(axis=0)
        X[n_clu:] = rng.uniform(lo, hi, size=(n_noise, d)).astype(np.float32)
    return _shuffle(rng, X)


# --------------------------------------------------------------------------
# Named workloads. Sizes and distributions follow the configurations the
# library is measured on; each is deterministic in its seed.
# --------------------------------------------------------------------------

def blobs_circle_5k() -> Workload:
    """5,000 x 8: four blobs plus a noisy circle; L2 lens, 20 intervals at
    30 % overlap, eps 0.6, minPts 5."""
    X = blobs_and_circle(seed=0)
    return Workload("blobs_circle_5k_d8", X, (LENS_L2,), (0,), (20,), (0.30,), 0.6, 5)


def mixture_100k(n: int = 100_000) -> Workload:
    """100,000 x 64: 16 anisotropic Gaussians; PC1 lens, 50 intervals at 25 %
    overlap, eps at the 2nd percentile of sampled distances, minPts 10."""
    X = gaussian_mixture(n, 64, 16, seed=1, centre_box=10.0, std_lo=0.3, std_hi=1.5,
                         anisotropic=True)
    eps = eps_at_percentile(X, 2.0, seed=1)
    return Workload(f"mixture_{n // 1000}k_d64", X, (LENS_PCA,), (0,), (50,), (0.25,), eps, 10)


def clusters_1m_d256(n: int = 1_000_000) -> Workload:
    """1,000,000 x 256 (paper scale): 32 isotropic Gaussians (std in [0.5, 2],
    centres in [-20, 20]^256) plus 5 % uniform noise; L2 lens, 100 intervals
    at 20 % overlap, eps at the 1st percentile of sampled distances, minPts 5."""
    X = gaussian_mixture(n, 256, 32, seed=2, centre_box=20.0, std_lo=0.5, std_hi=2.0,
                         anisotropic=False, noise_frac=0.05)
    eps = eps_at_percentile(X, 1.0, seed=2)
    return Workload(f"clusters_{n // 1000}k_d256", X, (LENS_L2,), (0,), (100,), (0.20,), eps, 5)


def zipf_mixture_500k(n: int = 500_000) -> Workload:
    """500,000 x 128: 24 anisotropic Gaussians with Zipf(1.2) weights; 2D lens
    (PC1, PC2) on a 30 x 30 grid at 25 % overlap; eps at the 1st percentile,
    minPts 10."""
    w = np.arange(1, 25, dtype=np.float64) ** -1.2
    X = gaussian_mixture(n, 128, 24, seed=3, centre_box=10.0, std_lo=0.3, std_hi=1.5,
                         anisotropic=True, weights=w)
    eps = eps_at_percentile(X, 1.0, seed=3)
    return Workload(f"zipf_mixture_{n // 1000}k_d128", X, (LENS_PCA, LENS_PCA), (0, 1),
                    (30, 30), (0.25, 0.25), eps, 10)


def circle(n: int = 600, phase: float = 0.0123) -> np.ndarray:
    """Evenly spaced points on the unit circle in the plane (no noise)."""
    t = phase + 2.0 * np.pi * np.arange(n) / n
    return np.stack([np.cos(t), np.sin(t)], axis=1).astype(np.float32)


def separated_blobs(k: int, per: int, d: int, gap: float, std: float, seed: int) -> np.ndarray:
    """k Gaussian blobs whose centres sit `gap` apart along a random direction
    family (centre c_i = i * gap * e_(i mod d)), shuffled."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(k):
        c = np.zeros(d)
        c[i % d] = gap * (1 + i // d)
        parts.append(c + std * rng.standard_normal((per, d)))
    return _shuffle(rng, np.concatenate(parts).astype(np.float32))


def tiny_random(n: int, d: int, seed: int, scale: float = 1.0, dup_frac: float = 0.0) -> np.ndarray:
    """Small uniform cloud in [0, scale]^d, optionally with duplicated rows."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, scale, size=(n, d)).astype(np.float32)
    n_dup = int(dup_frac * n)
    if n_dup:
        src = rng.integers(0, n, size=n_dup)
        dst = rng.integers(0, n, size=n_dup)
        X[dst] = X[src]
    return X


# --------------------------------------------------------------------------
# Serving mix: resident clouds and a seeded Poisson request stream.
# --------------------------------------------------------------------------

def pair_sample(X: np.ndarray, seed: int, n_pairs: int = 100_000) -> np.ndarray:
    """Sorted squared distances of n_pairs uniformly drawn pairs i != j."""
    rng = np.random.default_rng([seed, 0x5E7])
    n = X.shape[0]
    i = rng.integers(0, n, size=n_pairs)
    j = rng.integers(0, n - 1, size=n_pairs)
    j = j + (j >= i)
    sq = np.empty(n_pairs, dtype=np.float64)
    for s in range(0, n_pairs, 8192):
        diff = X[i[s:s + 8192]].astype(np.float64) - X[j[s:s + 8192]].astype(np.float64)
        sq[s:s + 8192] = np.einsum("ij,ij->i", diff, diff)
    sq.sort()
    return sq


def eps_from_sample(sq: np.ndarray, q: float) -> float:
    """Radius halfway (in squared distance) between the sampled values around
    the q-th percentile, as in eps_at_percentile."""
    k = min(max(int(math.ceil(q * len(sq) / 100.0)) - 1, 0), len(sq) - 2)
    return float(math.sqrt(0.5 * (sq[k] + sq[k + 1])))


def serving_datasets(seed: int = 4, big_n: int = 1_000_000, big_X: np.ndarray | None = None):
    """Nine resident clouds: the 1,000,000 x 256 clustered cloud and eight
    Gaussian mixtures (16 clusters) with n log-uniform in [1e4, 5e5] and d in
    {32, 64, 128, 256}. big_X: the clustered cloud, when already drawn."""
    rng = np.random.default_rng(seed)
    out = [clusters_1m_d256(big_n).X if big_X is None else big_X]
    for k in range(8):
        n = int(round(10 ** rng.uniform(4.0, math.log10(5e5))))
        d = int(rng.choice([32, 64, 128, 256]))
        out.append(gaussian_mixture(n, d, 16, seed=100 + k, centre_box=10.0, std_lo=0.3, std_hi=1.5,
                                    anisotropic=True))
    return out


def serving_requests(samples, n_requests: int, rate: float, seed: int = 4):
    """Poisson arrivals (mean `rate` per second); each request draws a
    dataset, lens in {L2, PC1}, n_intervals in [10, 200], overlap in
    [0.1, 0.5], eps at a percentile in [0.5, 4] and minPts in [3, 20].
    `samples` are the datasets' pair_sample arrays. Returns a list of dicts
    with arrival time `t` (seconds) and the mapper parameters."""
    rng = np.random.default_rng([seed, 0x5E4])
    t = 0.0
    reqs = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate)
        ds = int(rng.integers(0, len(samples)))
        lens = LENS_L2 if rng.random() < 0.5 else LENS_PCA
        reqs.append(dict(t=t, dataset=ds, lens_kind=(lens,), lens_arg=(0,),
                         n_intervals=(int(rng.integers(10, 201)),), overlap=(float(rng.uniform(0.1, 0.5)),),
                         eps=eps_from_sample(samples[ds], float(rng.uniform(0.5, 4.0))),
                         min_pts=int(rng.integers(3, 21))))
    return reqs


def zipf_sweep(n: int = 500_000):
    """The 2D-lens sweep: the Zipf(1.2) mixture of 24 clusters (n x 128),
    (PC1, PC2) lens on a 30 x 30 grid, minPts 10, and 16 (eps, overlap)
    points: eps at the 0.5/1/2/4th percentile of sampled distances times
    overlap 0.1/0.2/0.3/0.4. Returns (workload, eps list, overlap list)."""
    w = zipf_mixture_500k(n)
    sq = pair_sample(w.X, 3)
    eps, ov = [], []
    for q in (0.5, 1.0, 2.0, 4.0):
        for p in (0.1, 0.2, 0.3, 0.4):
            eps.append(eps_from_sample(sq, q))
            ov.append(p)
    return w, eps, ov
