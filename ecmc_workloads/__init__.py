"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no event-chain arithmetic: only the box geometry of the
hard-disk model (Sec. 2, eq. 1: eta = N pi sigma^2 / (4 L^2)), square-lattice
starting configurations, and the workload table the tests and the benchmark
use.  Both the CUDA library and the oracle receive what it produces as input.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ETA_HCP = math.pi / (2.0 * math.sqrt(3.0))


def box_side(N: int, eta: float, sigma: float = 1.0) -> float:
    """L = sigma sqrt(N pi / (4 eta)) (eq. 1 solved for L)."""
    return sigma * math.sqrt(N * math.pi / (4.0 * eta))


def box_side3(N: int, eta: float, sigma: float = 1.0) -> float:
    """Hard spheres: L = sigma (N pi / (6 eta))^(1/3), from
    eta = N pi sigma^3 / (6 L^3)."""
    return sigma * (N * math.pi / (6.0 * eta)) ** (1.0 / 3.0)


def cubic_lattice(N: int, L: float):
    """k x k x k simple cubic lattice, k = N^(1/3): sphere (iz*k + iy)*k + ix
    sits at ((ix + 1/2) a, (iy + 1/2) a, (iz + 1/2) a) with a = L / k."""
    k = int(round(N ** (1.0 / 3.0)))
    if k * k * k != N:
        raise ValueError("N=%d is not a perfect cube" % N)
    a = L / k
    i = np.arange(N, dtype=np.int64)
    x = ((i % k).astype(np.float64) + 0.5) * a
    y = (((i // k) % k).astype(np.float64) + 0.5) * a
    z = ((i // (k * k)).astype(np.float64) + 0.5) * a
    return np.ascontiguousarray(x), np.ascontiguousarray(y), np.ascontiguousarray(z)


def packing_fraction(N: int, L: float, sigma: float = 1.0) -> float:
    return N * math.pi * sigma * sigma / (4.0 * L * L)


def square_lattice(N: int, L: float):
    """k x k square lattice, k = sqrt(N): disk iy*k + ix sits at
    ((ix + 1/2) a, (iy + 1/2) a) with a = L / k.  Returns float64 x, y."""
    k = int(round(math.sqrt(N)))
    if k * k != N:
        raise ValueError("N=%d is not a perfect square" % N)
    a = L / k
    ix = np.arange(N, dtype=np.int64) % k
    iy = np.arange(N, dtype=np.int64) // k
    x = (ix.astype(np.float64) + 0.5) * a
    y = (iy.astype(np.float64) + 0.5) * a
    return np.ascontiguousarray(x), np.ascontiguousarray(y)


def random_gas(N: int, L: float, sigma: float, seed: int, max_tries: int = 200000):
    """Random sequential addition of N non-overlapping disks (low densities
    only): uniform trial centres from numpy's PCG64 with the given seed."""
    rng = np.random.default_rng(seed)
    pts = np.empty((N, 2))
    n = 0
    tries = 0
    while n < N:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random_gas: density too high for sequential addition")
        p = rng.random(2) * L
        if n:
            d = pts[:n] - p
            d -= L * np.round(d / L)
            if np.min(np.einsum("ij,ij->i", d, d)) < sigma * sigma:
                continue
        pts[n] = p
        n += 1
    return np.ascontiguousarray(pts[:, 0]), np.ascontiguousarray(pts[:, 1])


@dataclass
class Workload:
    name: str
    N: int
    eta: float
    cells: int
    ell: float
    seed: int
    sigma: float = 1.0
    sweeps: int = 0
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def L(self) -> float:
        return box_side(self.N, self.eta, self.sigma)

    def lattice(self):
        return square_lattice(self.N, self.L)


# The paper's workloads (Sec. 3.4 and Sec. 4: N = 256^2 at eta 0.698-0.718,
# N = 64^2 at 0.704) and the sizes used here, all started from square lattices.
SMALL = Workload("N=256 eta=0.70", 256, 0.70, 2, 4.0, seed=1, sweeps=1000)
MEDIUM = Workload("N=65536 eta=0.708", 65536, 0.708, 32, 8.0, seed=2,
                  sweeps=10000)
LARGE = Workload("N=1048576 eta=0.72", 1048576, 0.72, 128, 8.0, seed=3)
HUGE = Workload("N=4194304 eta=0.716", 4194304, 0.716, 256, 8.0, seed=5)

# Parallelisation grid at N = 1M, eta = 0.72: cells per side x ell.
LARGE_CELL_GRID = [8, 16, 32, 64, 128, 256, 512]
LARGE_ELL_GRID = [2.0, 8.0, 32.0]


def round_to_square(n: float) -> int:
    k = max(1, int(round(math.sqrt(n))))
    return k * k


def replica_batch(seed: int = 4, R: int = 96):
    """Many independent replicas of uneven size and density: N log-uniform in
    [4096, 262144] (u from numpy's Philox with key (seed, r)), rounded to a
    perfect square for the lattice start; eta = 0.600 + 0.005 (r mod 29).
    Returns a list of dicts with N, eta, L, seed, replica."""
    out = []
    for r in range(R):
        u = np.random.Generator(np.random.Philox(key=[seed, r])).random()
        N = round_to_square(4096.0 * 64.0**u)
        eta = 0.600 + 0.005 * (r % 29)
        out.append(dict(N=N, eta=eta, L=box_side(N, eta), seed=seed, replica=r))
    return out


def eos_batch(seed: int = 6, R: int = 32, N: int = 262144):
    """Equation-of-state batch: R replicas of N disks at packing fractions
    evenly spaced from 0.69 to 0.74."""
    etas = np.linspace(0.69, 0.74, R)
    return [dict(N=N, eta=float(e), L=box_side(N, float(e)), seed=seed, replica=r)
            for r, e in enumerate(etas)]
