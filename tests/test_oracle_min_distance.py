"""Pins of the oracle's smallest-pair-distance functions (the overlap check of
ecmc_set_positions and ecmc3_set_positions): the grid search must return,
bit for bit, the minimum over ALL pairs of the minimum-image squared
distance, or rcut^2 when no pair is closer than rcut, as a brute force over
every pair computes it with the same rounded operations.  Cases: random
points (the grid path and the all-pairs path for small boxes), a closest pair
across the periodic boundary, no pair within rcut, and melted dense
configurations."""
import numpy as np
import pytest

import ecmc_workloads as W
import oracle


def wrap(v, L):
    return np.where(v >= 0.5 * L, v - L, np.where(v < -0.5 * L, v + L, v))


def brute(L, rcut, *coords):
    n = coords[0].shape[0]
    iu = np.triu_indices(n, 1)
    d2 = np.zeros(len(iu[0]))
    for c in coords:
        d = wrap(c[iu[1]] - c[iu[0]], L)
        d2 = d2 + d * d
    m = d2.min() if d2.size else np.inf
    return min(m, rcut * rcut)


@pytest.mark.parametrize("N,L,rcut,seed", [(800, 40.0, 2.0, 1), (300, 5.0, 2.0, 2),
                                           (2000, 60.0, 1.5, 3), (2, 9.0, 2.0, 4)])
def test_two_dimensions_random_points(N, L, rcut, seed):
    rng = np.random.default_rng(seed)
    x, y = rng.random(N) * L, rng.random(N) * L
    assert oracle.min_dist2(L, x, y, rcut) == brute(L, rcut, x, y)


def test_two_dimensions_closest_pair_across_the_boundary():
    L = 30.0
    rng = np.random.default_rng(7)
    x, y = rng.random(50) * L, rng.random(50) * L
    x[0], y[0] = 0.05, 11.0
    x[1], y[1] = L - 0.07, 11.01
    got = oracle.min_dist2(L, x, y, 2.0)
    assert got == brute(L, 2.0, x, y) and abs(got - 0.0145) < 1e-12  # (0.12, 0.01) apart


def test_two_dimensions_no_pair_within_rcut():
    L = 100.0
    x = np.array([5.0, 50.0, 95.0 - 1e-9])
    y = np.array([5.0, 50.0, 50.0])
    assert oracle.min_dist2(L, x, y, 2.0) == 4.0  # 95 - 1e-9 is 10 - 1e-9 from 5 around the box


def test_two_dimensions_melted_dense_configuration():
    N, eta = 4096, 0.72
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, 16, 16, 1.0, 4, 9)
    oracle.sweeps(p, x, y, 0, 6)
    assert oracle.min_dist2(L, x, y, 2.0) == brute(L, 2.0, x, y)


@pytest.mark.parametrize("N,L,rcut,seed", [(600, 20.0, 2.0, 5), (150, 5.0, 2.0, 6)])
def test_three_dimensions_random_points(N, L, rcut, seed):
    rng = np.random.default_rng(seed)
    x, y, z = rng.random(N) * L, rng.random(N) * L, rng.random(N) * L
    assert oracle.min_dist2_3(L, x, y, z, rcut) == brute(L, rcut, x, y, z)


def test_three_dimensions_across_the_boundary_and_melted():
    N, eta = 1000, 0.45
    L = W.box_side3(N, eta)
    x, y, z = W.cubic_lattice(N, L)
    p = oracle.make_params3(N, L, 1.0, 4, 1.0, 3, 2)
    oracle.sweeps3(p, x, y, z, 0, 6)
    assert oracle.min_dist2_3(L, x, y, z, 2.0) == brute(L, 2.0, x, y, z)
    x[0], y[0], z[0] = 0.01, 0.02, L - 0.03
    x[1], y[1], z[1] = L - 0.02, 0.03, 0.04
    got = oracle.min_dist2_3(L, x, y, z, 2.0)
    assert got == brute(L, 2.0, x, y, z) and got < 0.01
