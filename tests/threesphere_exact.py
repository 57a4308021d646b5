"""Exact pair-distance distribution of three hard spheres in a periodic cube,
for distances below L/2.

For the uniform measure on non-overlapping configurations of three spheres
of diameter sigma in a periodic cube of side L (L > 2 sigma), fix sphere 1
at the origin (translation invariance).  The separation u of sphere 2 from
sphere 1 has the density

    p(u) ~ 1[|u|_min >= sigma] * V_free(u),
    V_free(u) = L^3 - 2 (4 pi / 3) sigma^3 + sum_k lens(|u + k L|),

the volume left to the centre of sphere 3: the cube minus the two exclusion
balls of radius sigma around spheres 1 and 2, whose overlap is the sum over
the periodic images k of u of the lens volume of two balls of radius sigma
at distance d, pi (4 sigma + d) (2 sigma - d)^2 / 12 for d < 2 sigma (two
images of one ball never overlap because L > 2 sigma).  For r = |u| < L/2
the whole sphere |u| = r lies inside the fundamental cube, so the marginal
density of the minimum-image distance there is r^2 times the integral of
V_free over the directions: smooth, integrated here with Gauss-Legendre
nodes in r and a Fibonacci lattice of directions.  All three pairs share
this marginal.
"""
import math

import numpy as np


def lens_volume(d, R):
    """Volume of the intersection of two balls of radius R at distance d."""
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    m = d < 2.0 * R
    dm = d[m]
    out[m] = math.pi * (4.0 * R + dm) * (2.0 * R - dm) ** 2 / 12.0
    return out


def free_volume(u, L, sigma):
    """V_free for separations u of shape (..., 3)."""
    v = np.full(u.shape[:-1], L**3 - 2.0 * (4.0 * math.pi / 3.0) * sigma**3)
    for kx in (-1, 0, 1):
        for ky in (-1, 0, 1):
            for kz in (-1, 0, 1):
                s = u + L * np.array([kx, ky, kz], dtype=np.float64)
                v = v + lens_volume(np.sqrt((s * s).sum(-1)), sigma)
    return v


def fibonacci_directions(n):
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = math.pi * (3.0 - math.sqrt(5.0)) * i
    rxy = np.sqrt(1.0 - z * z)
    return np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], 1)


def bin_probabilities(edges, L, sigma, n_dir=4000, n_r=12):
    """Probabilities of the bins [edges[i], edges[i+1]) of the minimum-image
    pair distance, conditional on sigma <= r < edges[-1] <= L/2."""
    assert edges[0] >= sigma and edges[-1] <= 0.5 * L and L > 2.0 * sigma
    dirs = fibonacci_directions(n_dir)
    xg, wg = np.polynomial.legendre.leggauss(n_r)
    p = np.empty(len(edges) - 1)
    for b in range(len(edges) - 1):
        a, c = edges[b], edges[b + 1]
        r = 0.5 * (c - a) * xg + 0.5 * (c + a)
        tot = 0.0
        for rk, wk in zip(r, wg):
            ang = free_volume(rk * dirs, L, sigma).mean() * 4.0 * math.pi
            tot += wk * rk * rk * ang
        p[b] = 0.5 * (c - a) * tot
    return p / p.sum()
