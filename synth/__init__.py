"""Seeded synthetic point clouds for the five workloads and for tests.

Shared by the tests, the oracle's callers and the benchmark.  This module
holds no step of the complex build: it only draws points (numpy PCG64, seed
1809 + workload index) and derives each workload's radius cap as a quantile of
pairwise squared distances -- a parameter of the input, computed here with
plain numpy (exactly for integers, blockwise Gram form or a pair sample for
floats).

The paper's datasets (Dragon, WorldMap, HIV, Klein, C. elegans) are not
available; these shapes stand in for them: a torus and a sphere in R^3 (like
the Dragon/WorldMap point sets) and Gaussian mixtures in higher dimension.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

I8, I32, F32 = 1, 2, 3


@dataclass
class Cloud:
    points: np.ndarray   # (n, d) int8 / int32 / float32, row-major
    maxdim: int
    maxrad: float

    @property
    def n(self) -> int:
        return self.points.shape[0]

    @property
    def d(self) -> int:
        return self.points.shape[1]

    @property
    def dtype_code(self) -> int:
        return {np.dtype(np.int8): I8, np.dtype(np.int32): I32,
                np.dtype(np.float32): F32}[self.points.dtype]


@dataclass
class Matrix:
    """A square symmetric matrix of edge values as the input."""
    points: np.ndarray   # (n, n) int32 / float32, row-major
    maxdim: int
    maxrad: float

    @property
    def n(self) -> int:
        return self.points.shape[0]

    @property
    def d(self) -> int:
        return 0

    @property
    def dtype_code(self) -> int:
        return {np.dtype(np.int32): I32, np.dtype(np.float32): F32}[self.points.dtype]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def quantize(x: np.ndarray, scale: float) -> np.ndarray:
    """Scale, round half to even, clamp to [-127, 127], int8."""
    return np.clip(np.rint(x * scale), -127, 127).astype(np.int8)


def radius_above(d2: float) -> float:
    """A double r, just above sqrt(d2), with fl(r*r) >= d2: an inclusive cap
    at r keeps every pair with squared distance <= d2."""
    r = math.sqrt(d2)
    while r * r < d2:
        r = math.nextafter(r, math.inf)
    return math.nextafter(r, math.inf)


def _pair_d2_int(p: np.ndarray) -> np.ndarray:
    q = p.astype(np.int64)
    n = q.shape[0]
    iu = np.triu_indices(n, 1)
    out = np.zeros(iu[0].shape[0], dtype=np.int64)
    for k in range(q.shape[1]):
        t = q[iu[0], k] - q[iu[1], k]
        out += t * t
    return out


def _sampled_pair_d2(p: np.ndarray, g: np.random.Generator, m: int) -> np.ndarray:
    n = p.shape[0]
    i = g.integers(0, n, size=m)
    j = g.integers(0, n - 1, size=m)
    j = j + (j >= i)
    q = p.astype(np.float64)
    return np.sum((q[i] - q[j]) ** 2, axis=1)


# ----------------------------------------------------------------- workloads

def torus(n: int, g: np.random.Generator, R=3.0, r=1.0, sigma=0.05) -> np.ndarray:
    """Angle-uniform torus samples in R^3 plus Gaussian noise."""
    u = g.uniform(0.0, 2 * math.pi, n)
    v = g.uniform(0.0, 2 * math.pi, n)
    x = np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u),
                  r * np.sin(v)], axis=1)
    return x + g.normal(0.0, sigma, x.shape)


def sphere(n: int, g: np.random.Generator, sigma=0.02, d=3) -> np.ndarray:
    """Normalised Gaussian directions (unit sphere) plus Gaussian noise."""
    x = g.normal(size=(n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x + g.normal(0.0, sigma, x.shape)


def gaussian_mixture(n: int, d: int, g: np.random.Generator, k=8, box=5.0, sigma=1.0):
    centres = g.uniform(-box, box, size=(k, d))
    labels = g.integers(0, k, size=n)
    return (centres[labels] + g.normal(0.0, sigma, size=(n, d))).astype(np.float32)


def config1() -> Cloud:
    """n=64, d=3 int32 uniform in [-100, 100], no cap, maxdim 2."""
    g = rng(1809 + 1)
    return Cloud(g.integers(-100, 101, size=(64, 3)).astype(np.int32), 2, math.inf)


def config2(n: int = 1000) -> Cloud:
    """Torus (R=3, r=1) + N(0, 0.05^2), scale 30 -> int8; cap at the integer
    d^2 of rank floor(0.15 (N-1)) among all N pairs; maxdim 2."""
    g = rng(1809 + 2)
    p = quantize(torus(n, g), 30.0)
    d2 = np.sort(_pair_d2_int(p))
    cap2 = int(d2[int(math.floor(0.15 * (d2.shape[0] - 1)))])
    return Cloud(p, 2, radius_above(float(cap2)))


def config3(n: int = 4000, d: int = 32, maxdim: int = 2) -> Cloud:
    """Mixture of 8 Gaussians (centres uniform in [-5,5]^d, sigma 1), float32;
    cap at the 5th percentile of pairwise squared distance; maxdim 2."""
    g = rng(1809 + 3)
    p = gaussian_mixture(n, d, g)
    q = p.astype(np.float64)
    sq = np.sum(q * q, axis=1)
    vals = []
    for s in range(0, n, 512):
        blk = sq[s:s + 512, None] + sq[None, :] - 2.0 * (q[s:s + 512] @ q.T)
        ii = np.arange(s, min(s + 512, n))[:, None]
        jj = np.arange(n)[None, :]
        vals.append(blk[jj > ii])
    d2 = np.concatenate(vals)
    k = int(0.05 * (d2.shape[0] - 1))
    cap2 = float(np.partition(d2, k)[k])
    return Cloud(p, maxdim, radius_above(cap2))


def config4(n_clouds: int = 4096) -> list:
    """Uneven batch: sizes uniform in [32, 512], unit-sphere samples + N(0,
    0.02^2), scale 100 -> int8, cap 40 grid units (0.4 of the radius)."""
    g = rng(1809 + 4)
    sizes = g.integers(32, 513, size=n_clouds)
    return [Cloud(quantize(sphere(int(m), g), 100.0), 2, 40.0) for m in sizes]


def config5_request(g: np.random.Generator) -> Cloud:
    """One serving request: n log-uniform in [50, 5000]; half int8 d=3 (torus
    scale 30 or sphere scale 100), half float32 Gaussian mixtures at d=16;
    maxdim uniform in {1, 2}; cap at the pairwise-d^2 quantile
    q = clamp(k/n, 0.01, 0.15) with k ~ U[20, 100] (estimated from 4000
    sampled pairs)."""
    n = int(round(math.exp(g.uniform(math.log(50), math.log(5000)))))
    kind = g.integers(0, 4)
    if kind == 0:
        p = quantize(torus(n, g), 30.0)
    elif kind == 1:
        p = quantize(sphere(n, g), 100.0)
    else:
        p = gaussian_mixture(n, 16, g)
    maxdim = int(g.integers(1, 3))
    q = min(max(g.uniform(20, 100) / n, 0.01), 0.15)
    d2 = _sampled_pair_d2(p, g, 4000)
    cap2 = float(np.quantile(d2, q))
    if p.dtype == np.int8:
        cap2 = float(math.floor(cap2))
    return Cloud(p, maxdim, radius_above(cap2))


def config5(n_requests: int = 20000, rate_per_s: float = 1000.0, seed: int = 1809 + 5):
    """Poisson arrival times (seconds) and the requests, in arrival order."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_per_s, size=n_requests)
    return np.cumsum(gaps), [config5_request(g) for _ in range(n_requests)]


# ----------------------------------------------------------------- test clouds

def worldmap(n: int = 7322, maxdim: int = 2, seed: int = 1809 + 6) -> Cloud:
    """WorldMap-shaped single cloud: n = 7322 float32 points on the unit
    sphere, cap 0.15 (the paper's WorldMap run).  The city coordinates are
    not available; the stand-in clusters like land masses: 70 % of the points
    from 7 blobs (centres uniform on the sphere, N(0, 0.25^2) offsets,
    projected back to the sphere), 30 % uniform on the sphere."""
    g = rng(seed)
    k = 7
    centres = g.normal(size=(k, 3))
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    m = int(round(0.7 * n))
    lab = g.integers(0, k, size=m)
    a = centres[lab] + g.normal(scale=0.25, size=(m, 3))
    b = g.normal(size=(n - m, 3))
    p = np.concatenate([a, b])
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    p = p[g.permutation(n)]
    return Cloud(p.astype(np.float32), maxdim, 0.15)


def hamming_matrix(n: int = 1088, L: int = 1000, n_types: int = 9, seed: int = 1809 + 7):
    """HIV-shaped distance matrix: Hamming distances (int32) between n
    sequences of length L over 4 letters with subtype structure -- a random
    root, n_types subtypes each differing from it at 15 % of sites, each
    sequence differing from its subtype at 5 % of sites.  The paper's 1088
    HIV genomic sequences are not available."""
    g = rng(seed)
    root = g.integers(0, 4, size=L)
    types = np.repeat(root[None, :], n_types, axis=0)
    mut = g.random((n_types, L)) < 0.15
    types[mut] = (types[mut] + g.integers(1, 4, size=mut.sum())) % 4
    lab = g.integers(0, n_types, size=n)
    seqs = types[lab].copy()
    mut = g.random((n, L)) < 0.05
    seqs[mut] = (seqs[mut] + g.integers(1, 4, size=mut.sum())) % 4
    D = np.zeros((n, n), np.int32)
    for i in range(n):
        D[i] = (seqs != seqs[i]).sum(1)
    return D


def hiv(maxdim: int = 2) -> Matrix:
    """HIV-shaped workload: the 1088 x 1088 Hamming matrix, cap at its 10th
    percentile (59,846 edges, 2,106,840 triangles, 51 grades)."""
    D = hamming_matrix()
    return Matrix(D, maxdim, hamming_cap(D, 0.1))


def hamming_cap(D: np.ndarray, q: float) -> float:
    """The q-quantile of the strict-upper-triangle values (an integer)."""
    iu = np.triu_indices(D.shape[0], 1)
    return float(np.quantile(D[iu], q, method="lower"))


def random_cloud(n: int, d: int, dtype, seed: int, lo=-100, hi=100) -> np.ndarray:
    g = rng(seed)
    if np.dtype(dtype) == np.float32:
        return g.uniform(lo, hi, size=(n, d)).astype(np.float32)
    return g.integers(lo, hi + 1, size=(n, d)).astype(dtype)


def ngon(n: int, radius: float = 1.0) -> np.ndarray:
    t = 2 * math.pi * np.arange(n) / n
    return np.stack([radius * np.cos(t), radius * np.sin(t)], axis=1).astype(np.float32)


def circle_samples(n: int, seed: int) -> np.ndarray:
    """n points on the unit circle at sorted uniform angles (float32)."""
    g = rng(seed)
    t = np.sort(g.uniform(0.0, 2 * math.pi, n))
    return np.stack([np.cos(t), np.sin(t)], axis=1).astype(np.float32)
