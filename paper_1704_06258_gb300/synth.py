"""Seeded synthetic USApHMP instances and populations.

This module only draws inputs: node coordinates, the flow matrix W, the cost
matrix C (Euclidean distances, the metric setting of the paper's Urand and AP
families, §6.1) and random valid chromosomes in the (H, S) encoding of §4.1.
It contains none of the method's arithmetic (no cost, no allocation rule, no
GA operator), so both the FP64 oracle and the CUDA path can take their inputs
from it.

Every instance is FP32 (W and C are the instance; the oracle widens them to
FP64 exactly).  W_ii = 0 everywhere, and C is exactly symmetric with a zero
diagonal because each distance is computed once in FP64 from the coordinate
difference and then rounded to FP32.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CHI, ALPHA, DELTA = 3.0, 0.75, 2.0   # collection, transfer, distribution factors


@dataclasses.dataclass
class Instance:
    name: str
    n: int
    p: int
    W: np.ndarray        # float32 [n, n], row-major, W[i, j] = flow i -> j
    C: np.ndarray        # float32 [n, n], C[i, k] = unit cost of arc (i, k)
    chi: float = CHI
    alpha: float = ALPHA
    delta: float = DELTA
    xy: np.ndarray | None = None


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _euclid_fp32(xy: np.ndarray) -> np.ndarray:
    d = xy[:, None, :] - xy[None, :, :]
    C = np.sqrt(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1])
    return C.astype(np.float32)


def _zero_diag(W: np.ndarray) -> np.ndarray:
    np.fill_diagonal(W, 0.0)
    return W


def uniform_points(rng, n, side):
    return rng.uniform(0.0, side, size=(n, 2))


def clustered_points(rng, n, side=10000.0, k=8, sigma=50.0):
    centres = rng.uniform(0.0, side, size=(k, 2))
    which = rng.integers(0, k, size=n)
    xy = centres[which] + rng.normal(0.0, sigma, size=(n, 2))
    return np.clip(xy, 0.0, side)


def tiny(seed: int = 1001, n: int = 10, p: int = 3) -> Instance:
    """n=10, p=3; coordinates uniform in [0,100]^2; W uniform [0,1)."""
    rng = _rng(seed)
    xy = uniform_points(rng, n, 100.0)
    W = _zero_diag(rng.uniform(0.0, 1.0, size=(n, n)).astype(np.float32))
    return Instance(f"tiny_n{n}_p{p}", n, p, W, _euclid_fp32(xy), xy=xy)


def urand200(seed: int = 1002, n: int = 200, p: int = 10) -> Instance:
    """n=200; coordinates uniform in [0,1000]^2; W lognormal(0, 1)."""
    rng = _rng(seed)
    xy = uniform_points(rng, n, 1000.0)
    W = _zero_diag(rng.lognormal(0.0, 1.0, size=(n, n)).astype(np.float32))
    return Instance(f"urand_n{n}_p{p}", n, p, W, _euclid_fp32(xy), xy=xy)


def clustered(seed: int = 1003, n: int = 1000, p: int = 20) -> Instance:
    """8 Gaussian clusters (sigma 50) in [0,10^4]^2; W lognormal(0, 1.5)."""
    rng = _rng(seed)
    xy = clustered_points(rng, n)
    W = _zero_diag(rng.lognormal(0.0, 1.5, size=(n, n)).astype(np.float32))
    return Instance(f"clustered_n{n}_p{p}", n, p, W, _euclid_fp32(xy), xy=xy)


def large_uniform(seed: int = 1004, n: int = 6000, p: int = 20) -> Instance:
    """Coordinates uniform in [0,10^4]^2; W uniform [0,100) with 10% zeros."""
    rng = _rng(seed)
    xy = uniform_points(rng, n, 10000.0)
    W = rng.uniform(0.0, 100.0, size=(n, n)).astype(np.float32)
    W[rng.random(size=(n, n)) < 0.1] = 0.0
    return Instance(f"uniform_n{n}_p{p}", n, p, _zero_diag(W), _euclid_fp32(xy), xy=xy)


def latency_like(seed: int = 1005, n: int = 200, p: int = 10, spread: float = 0.6) -> Instance:
    """Non-metric costs standing in for the PlanetLab latencies of §6.1:
    coordinates uniform in [0,1000]^2, each Euclidean distance multiplied by
    a lognormal(0, spread) factor drawn once per unordered pair (so C stays
    symmetric with a zero diagonal but violates the triangle inequality on
    many triples); W lognormal(0, 1)."""
    rng = _rng(seed)
    xy = uniform_points(rng, n, 1000.0)
    d = xy[:, None, :] - xy[None, :, :]
    E = np.sqrt(d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1])
    f = rng.lognormal(0.0, spread, size=(n, n))
    f = np.triu(f, 1)
    f = f + f.T
    C = (E * f).astype(np.float32)
    W = _zero_diag(rng.lognormal(0.0, 1.0, size=(n, n)).astype(np.float32))
    return Instance(f"latency_n{n}_p{p}", n, p, W, _zero_diag(C), xy=xy)


def serving_request(r: int):
    """Request r of the serving mix: n log-uniform in [50, 3000], p in 3..20,
    instance drawn like the clustered family from seed 5000 + r."""
    rng = _rng(5000 + r)
    n = int(round(math.exp(rng.uniform(math.log(50.0), math.log(3000.0)))))
    p = int(rng.integers(3, 21))
    inst = clustered(seed=5000 + r, n=n, p=min(p, n))
    inst.name = f"request{r}_n{n}_p{inst.p}"
    return inst


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 4242) -> np.ndarray:
    """Arrival times (seconds from start) of a Poisson process."""
    rng = _rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def random_population(seed: int, n: int, p: int, B: int, nearest_like: bool = False):
    """B random valid chromosomes in the paper's encoding (§4.1).

    Returns (hubs int32 [B, p] node ids in random order, S int32 [B, n] node
    ids) with S[k] = k for every hub k and S[i] an open hub for every spoke.
    The allocation of spokes is uniform over the open hubs: it is any valid
    single allocation, not the nearest one.
    """
    rng = _rng(seed)
    hubs = np.empty((B, p), dtype=np.int32)
    S = np.empty((B, n), dtype=np.int32)
    for b in range(B):
        hb = rng.choice(n, size=p, replace=False).astype(np.int32)
        hubs[b] = hb
        S[b] = hb[rng.integers(0, p, size=n)]
        S[b, hb] = hb
    return hubs, S


def random_masks(seed: int, n: int, p: int, count: int) -> np.ndarray:
    """`count` boolean hub masks of length n with exactly p ones."""
    rng = _rng(seed)
    m = np.zeros((count, n), dtype=bool)
    for r in range(count):
        m[r, rng.choice(n, size=p, replace=False)] = True
    return m


CONFIGS = {
    "tiny": tiny,
    "urand200": urand200,
    "clustered1000": clustered,
    "uniform6000": large_uniform,
}
