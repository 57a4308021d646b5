"""Pins of the oracle's isotropic chain directions (the paper's preferred
mode for its applications, Sec. 4): a single disk at the centre of a large
cell, moved by one chain of budget ell per sweep with no wall in reach,
ends exactly at x0 + ell d, with d recomputed here from numpy's Philox4x64
by the rule the oracle states (the first Philox pair (u, v), uniform on
[-1, 1)^2, inside the unit disc, divided by its length); and the angles of
the oracle's displacements are uniform on the circle.  (A direction law that
is symmetric but not uniform would still sample the uniform measure, so the
three-disk test cannot see this.)
"""
import math

import numpy as np

import oracle
from test_oracle_draws import numpy_philox, unit

L, ELL, SEED, REPLICA = 20.0, 0.5, 21, 4


def iso_direction(t, c, k):
    for attempt in range(64):
        q = numpy_philox([t, 3, c, (k << 32) | attempt], [SEED, REPLICA])
        for h in (0, 1):
            u = 2.0 * unit(q[2 * h]) - 1.0
            v = 2.0 * unit(q[2 * h + 1]) - 1.0
            n2 = u * u + v * v
            if 0.0 < n2 <= 1.0:
                n = math.sqrt(n2)
                return u / n, v / n
    raise AssertionError("no point inside the disc")


def displacement(t):
    # one disk at the centre of cell 0 of a 2 x 2 grid without shift; the
    # walls are 5 away, the budget 0.5
    p = oracle.make_params(1, L, 1.0, 2, 2, ELL, 1, SEED, REPLICA,
                           dir_mode=oracle.DIR_ISOTROPIC, flags=oracle.FLAG_NO_SHIFT)
    x, y = np.array([5.0]), np.array([5.0])
    st, _ = oracle.sweeps(p, x, y, t, 1)
    assert st.events == 0 and st.wall_hits == 0 and st.chains == 1
    return x[0], y[0]


def test_direction_follows_the_stated_rule_bit_for_bit():
    for t in list(range(40)) + [1000, 123456, 2**33 + 7]:
        dx, dy = iso_direction(t, 0, 0)
        x, y = displacement(t)
        assert x == 5.0 + ELL * dx and y == 5.0 + ELL * dy
        assert abs(dx * dx + dy * dy - 1.0) < 4e-16


def test_angles_are_uniform_on_the_circle():
    n, nb = 36000, 36
    ang = np.empty(n)
    for t in range(n):
        x, y = displacement(t)
        ang[t] = math.atan2(y - 5.0, x - 5.0)
    hist = np.histogram(ang, bins=nb, range=(-math.pi, math.pi))[0]
    chi2 = np.sum((hist - n / nb) ** 2 / (n / nb))
    assert chi2 < 70.0  # 35 degrees of freedom, p ~ 5e-4
    # no preference for the axes or the diagonals: mean of cos 4 theta ~ 0
    assert abs(np.mean(np.cos(4 * ang))) < 4.0 * math.sqrt(0.5 / n)
    assert abs(np.mean(np.cos(ang))) < 4.0 * math.sqrt(0.5 / n)
