"""The pressure route through the contact value of g(r) (eq. pressure:
beta P / rho = 1 + (pi/2) rho sigma^2 g(sigma+)), with g(sigma+) the
quadratic least-squares fit over the first five 0.01 sigma bins evaluated at
sigma (the reading used for the rejecting boundary rule, whose pressure the
collision estimator does not give).  At eta = 0.1 the virial series
(tests/golden/hard_disk_virial.txt) fixes the answer; the oracle's g(r) must
reach it through this route for the reflecting and for the rejecting rule
(which samples the same uniform measure when starts are drawn with
replacement)."""
import math
import os

import numpy as np
import pytest

import ecmc_workloads as W
import oracle
from bench import contact_value

HERE = os.path.dirname(os.path.abspath(__file__))


def virial_golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "hard_disk_virial.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


@pytest.mark.parametrize("boundary", [oracle.BOUNDARY_REFLECT, oracle.BOUNDARY_REJECT])
def test_contact_value_route_matches_virial_series(boundary):
    N, eta, dr, nb = 400, 0.10, 0.01, 20
    L = W.box_side(N, eta)
    rho = N / L**2
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, 4, 4, 2.0, 10, 3, boundary=boundary)
    oracle.sweeps(p, x, y, 0, 200)
    t, vals = 200, []
    for _ in range(10):
        counts = np.zeros(nb, np.int64)
        for _ in range(400):
            oracle.sweeps(p, x, y, t, 1)
            t += 1
            counts += oracle.gr_counts(L, x, y, 1.0, dr, nb)
        R, g = oracle.gr_normalise(counts.astype(float), 400, N, L, 1.0, dr)
        vals.append(1.0 + 0.5 * math.pi * rho * contact_value(R, g))  # beta P / rho
    v = np.array(vals)
    z, se = v.mean(), v.std(ddof=1) / math.sqrt(len(v))
    gv = virial_golden()
    x2 = 0.5 * math.pi * rho  # B2 rho
    vir = 1.0 + x2 + gv["B3_over_B2sq"] * x2**2 + gv["B4_over_B2cu"] * x2**3
    assert abs(z - vir) < 4.0 * se + 1e-3, (z, vir, se)
