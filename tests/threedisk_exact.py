"""Exact pair-distance distribution of three hard disks in a periodic box.

For the uniform measure on non-overlapping configurations of three disks of
diameter sigma in a periodic L x L box (L > 2 sigma), fix disk 1 at the
origin (translation invariance).  The separation u of disk 2 from disk 1 has
the density

    p(u) ~ 1[|u|_min >= sigma] * A_free(u),
    A_free(u) = L^2 - 2 pi sigma^2 + sum_k lens(|u + k L|),

where A_free is the area left to the centre of disk 3 on the torus: the box
minus the two exclusion discs of radius sigma around disks 1 and 2, whose
overlap is the sum of the lens areas over the periodic images k of u (two
images of one disc never overlap each other because L > 2 sigma).  The
minimum-image distance r = |u|_min is then integrated over the arcs of the
circle |u| = r inside the fundamental cell [-L/2, L/2)^2, using the 8-fold
symmetry of the square.  All three pairs share this marginal.
"""
import math

import numpy as np


def lens_area(d, R):
    """Area of the intersection of two discs of radius R at distance d."""
    d = np.asarray(d, dtype=np.float64)
    out = np.zeros_like(d)
    m = d < 2.0 * R
    dm = d[m]
    out[m] = 2.0 * R * R * np.arccos(dm / (2.0 * R)) - 0.5 * dm * np.sqrt(4.0 * R * R - dm * dm)
    return out


def free_area(ux, uy, L, sigma):
    a = np.full(np.broadcast(ux, uy).shape, L * L - 2.0 * math.pi * sigma * sigma)
    for kx in (-1, 0, 1):
        for ky in (-1, 0, 1):
            d = np.hypot(ux + kx * L, uy + ky * L)
            a = a + lens_area(d, sigma)
    return a


def bin_probabilities(edges, L, sigma, n_r=16, n_theta=512):
    """Probability of the minimum-image pair distance falling in each bin
    [edges[i], edges[i+1]).  Gauss-Legendre quadrature in r on pieces between
    the kinks of the integrand (sigma, 2 sigma, L/2, the bin edges) and in
    theta over the arc of the circle |u| = r inside the first octant of the
    fundamental cell; normalised over [sigma, L/sqrt(2)]."""
    rmax = L / math.sqrt(2.0)
    xg, wg = np.polynomial.legendre.leggauss(n_r)
    xt, wt = np.polynomial.legendre.leggauss(n_theta)
    knots = sorted(set([sigma, 2.0 * sigma, L / 2.0, rmax] +
                       [e for e in edges if sigma <= e <= rmax]))
    piece = {}
    for a, b in zip(knots[:-1], knots[1:]):
        vals = []
        for r in 0.5 * (b - a) * xg + 0.5 * (b + a):
            c = L / (2.0 * r)
            lo = 0.0 if c >= 1.0 else math.acos(c)
            hi = math.pi / 4.0
            th = 0.5 * (hi - lo) * xt + 0.5 * (hi + lo)
            arc = 0.5 * (hi - lo) * np.sum(wt * free_area(r * np.cos(th), r * np.sin(th), L, sigma))
            vals.append(8.0 * r * arc)
        piece[(a, b)] = 0.5 * (b - a) * float(np.dot(wg, vals))
    total = sum(piece.values())
    out = []
    for e0, e1 in zip(edges[:-1], edges[1:]):
        out.append(sum(v for (a, b), v in piece.items() if a >= e0 - 1e-15 and b <= e1 + 1e-15))
    return np.array(out) / total
