"""Seeded synthetic TSP instances shaped like the benchmark sets of the paper.

The paper measures on TSPLIB instances from att48 to pr2392 (Section IV,
Tables 2-4).  Those files are not shipped here; these generators stand in for
them with the same city counts and coordinate statistics.  Everything in this
module is input preparation (coordinates and the rounded integer distance
matrix), shared by the CUDA path and by the CPU oracle; none of the Ant System
arithmetic lives here.

Distances follow the usual TSPLIB EUC_2D convention: the Euclidean distance
rounded to the nearest integer, ``floor(sqrt(dx^2 + dy^2) + 0.5)``.  The square
root of an integer is never exactly k + 1/2, so there is no rounding tie.
Duplicate coordinates are redrawn so that every off-diagonal distance is >= 1
(eta = 1/d is then always defined, Section II).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


class Instance:
    """One symmetric TSP instance: int64 coordinates; the int32 distance matrix
    (symmetric, zero diagonal, >= 1 elsewhere) is built on first use."""

    def __init__(self, coords: np.ndarray, kind: str, seed: int):
        self.coords = coords  # (n, 2) int64
        self.kind = kind
        self.seed = seed
        self._dist = None

    @property
    def dist(self) -> np.ndarray:
        if self._dist is None:
            self._dist = distance_matrix(self.coords)
        return self._dist

    @property
    def n(self) -> int:
        return int(self.coords.shape[0])


def distance_matrix(coords: np.ndarray) -> np.ndarray:
    """Rounded Euclidean distances (TSPLIB EUC_2D) as a C-contiguous int32 matrix."""
    c = np.asarray(coords, dtype=np.float64)
    dx = c[:, None, 0] - c[None, :, 0]
    dy = c[:, None, 1] - c[None, :, 1]
    d = np.floor(np.sqrt(dx * dx + dy * dy) + 0.5)
    return np.ascontiguousarray(d.astype(np.int32))


def _dedupe(coords: np.ndarray, redraw) -> np.ndarray:
    """Redraw rows that repeat an earlier row until all rows are distinct."""
    coords = coords.copy()
    while True:
        _, first = np.unique(coords, axis=0, return_index=True)
        dup = np.setdiff1d(np.arange(len(coords)), first)
        if dup.size == 0:
            return coords
        coords[dup] = redraw(dup.size)


def uniform_instance(n: int, side: int, seed: int) -> Instance:
    """n cities with integer coordinates drawn uniformly from [0, side]^2."""
    if n < 1:
        raise ValueError("n must be positive")
    if n > (side + 1) ** 2:
        raise ValueError("not enough distinct grid points")
    rng = np.random.Generator(np.random.PCG64(seed))
    draw = lambda k: rng.integers(0, side + 1, size=(k, 2), dtype=np.int64)
    coords = _dedupe(draw(n), draw)
    return Instance(coords, "uniform", seed)


def clustered_instance(n: int, seed: int, clusters: int = 64, sigma: float = 300.0,
                       side: int = 20000) -> Instance:
    """n cities around `clusters` Gaussian centres.

    Centres are uniform reals in [0, side]^2; each city picks a centre uniformly
    and is offset by N(0, sigma^2) per axis, then rounded to the integer grid and
    clamped to [0, side].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(0.0, float(side), size=(clusters, 2))

    def draw(k: int) -> np.ndarray:
        which = rng.integers(0, clusters, size=k)
        pts = centres[which] + rng.normal(0.0, sigma, size=(k, 2))
        return np.clip(np.rint(pts), 0, side).astype(np.int64)

    coords = _dedupe(draw(n), draw)
    return Instance(coords, "clustered", seed)


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """`count` city counts n = round(exp(U(ln lo, ln hi))), seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(math.log(lo), math.log(hi), size=count)
    return np.clip(np.rint(np.exp(u)), lo, hi).astype(np.int64)


# ---------------------------------------------------------------------------
# The five workload recipes (sizes, seeds and parameters in one place).
# ---------------------------------------------------------------------------

AS_PARAMS = dict(alpha=1.0, beta=2.0, rho=0.5)


def workload_n48() -> dict:
    """Single instance, 48 uniform cities in [0,1000]^2, m = 48, 100 iterations."""
    inst = uniform_instance(48, 1000, seed=1)
    return dict(name="as-n48-uniform", inst=inst, m=48, iterations=100, seed=1, **AS_PARAMS)


def workload_n1002() -> dict:
    """Single instance, 1002 uniform cities in [0,10000]^2, m = 1002, 50 iterations."""
    inst = uniform_instance(1002, 10000, seed=2)
    return dict(name="as-n1002-uniform", inst=inst, m=1002, iterations=50, seed=2, **AS_PARAMS)


def workload_n2392() -> dict:
    """Single instance, 2392 clustered cities (64 clusters, sigma 300, [0,20000]^2), m = 2392, 20 iterations."""
    inst = clustered_instance(2392, seed=3)
    return dict(name="as-n2392-clustered", inst=inst, m=2392, iterations=20, seed=3, **AS_PARAMS)


def workload_batched(count: int = 256) -> dict:
    """`count` independent uniform instances, n log-uniform in [48, 1024], m = n, 100 iterations.

    Instance i uses coordinate seed 1000 + i and Philox seed 1000 + i.
    """
    ns = log_uniform_sizes(count, 48, 1024, seed=4)
    insts = [uniform_instance(int(n), 1000, seed=1000 + i) for i, n in enumerate(ns)]
    return dict(name=f"as-batched-{count}", insts=insts, ms=[int(n) for n in ns],
                seeds=[1000 + i for i in range(count)], iterations=100, **AS_PARAMS)


def served_request(r: int, nmin: int = 48, nmax: int = 4096) -> dict:
    """Request r of the served stream: n log-uniform in [nmin, nmax], uniform or clustered 50/50.

    m = min(n, 1024), 200 iterations, Philox seed 10^6 + r.
    """
    rng = np.random.Generator(np.random.PCG64(10**6 + r))
    n = int(np.clip(np.rint(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))), nmin, nmax))
    if rng.uniform() < 0.5:
        inst = uniform_instance(n, 1000, seed=10**6 + r)
    else:
        inst = clustered_instance(n, seed=10**6 + r)
    return dict(inst=inst, m=min(n, 1024), iterations=200, seed=10**6 + r, **AS_PARAMS)


def poisson_arrivals(rate: float, duration: float, seed: int = 5) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream with the given rate over [0, duration)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    times = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return np.asarray(times)
        times.append(t)
