"""The pressure route through the contact value of g(r) (eq. pressure:
beta P / rho = 1 + (pi/2) rho sigma^2 g(sigma+)), with g(sigma+) the
quadratic least-squares fit over the first five 0.01 sigma bins evaluated at
sigma (the reading used for the rejecting boundary rule, whose pressure the
collision estimator does not give).  At eta = 0.1 the virial series
(tests/golden/hard_disk_virial.txt) fixes the answer; the oracle's g(r) must
reach it through this route for the reflecting and for the rejecting rule
(which samples the same uniform measure when starts are drawn with
replacement).  At eta = 0.6, where g(r) falls steeply from contact, the route
is pinned to the collision estimator (itself pinned to the virial series and
to the sequential chain) on the same run, and across the two rules."""
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


def contact_and_collision_batches(eta, boundary, ell, n_m, n_batches=10, per_batch=1000,
                                  N=256, cells=4, dr=0.01, nb=20, seed=11):
    """Both pressure estimators on one oracle run, batch by batch: the
    member-weighted collision sums and the contact value of g(r) measured
    every two sweeps."""
    L = W.box_side(N, eta)
    rho = N / L**2
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, cells, cells, ell, n_m, seed, boundary=boundary)
    oracle.sweeps(p, x, y, 0, 500)
    t, coll, cont = 500, [], []
    for _ in range(n_batches):
        counts = np.zeros(nb, np.int64)
        sb = sd = 0.0
        for _ in range(per_batch):
            st, _ = oracle.sweeps(p, x, y, t, 2)
            t += 2
            sb, sd = sb + st.sum_b_w, sd + st.sum_disp_w
            counts += oracle.gr_counts(L, x, y, 1.0, dr, nb)
        R, g = oracle.gr_normalise(counts.astype(float), per_batch, N, L, 1.0, dr)
        cont.append(1.0 + 0.5 * math.pi * rho * contact_value(R, g))
        coll.append(1.0 + sb / sd)
    return np.array(coll), np.array(cont)


def test_dense_contact_route_matches_collision_estimator():
    # at eta = 0.6 (beta P / rho ~ 6.5, g(sigma+) ~ 4.6, steep near contact)
    # the two routes to eq. (pressure) agree on the same run; a factor pi
    # for pi / 2 fails, and so does g read off the first bin without the
    # extrapolation to contact (0.14 low, 5 standard errors)
    coll, cont = contact_and_collision_batches(0.60, oracle.BOUNDARY_REFLECT, 4.0, 1)
    d = cont - coll
    se = d.std(ddof=1) / math.sqrt(len(d))
    assert abs(d.mean()) < 4.0 * se, (coll.mean(), cont.mean(), se)
    assert 6.0 < coll.mean() < 7.0


def test_dense_rejecting_rule_contact_pressure_matches_reflecting_rule():
    # the rejecting rule samples the same measure, so its pressure from
    # g(sigma+) equals the reflecting rule's collision pressure; its own
    # collision sums do not (they count only the chains that were kept, a
    # subset biased towards chains with few collisions)
    coll_ref, _ = contact_and_collision_batches(0.60, oracle.BOUNDARY_REFLECT, 4.0, 1)
    coll_rej, cont_rej = contact_and_collision_batches(0.60, oracle.BOUNDARY_REJECT, 0.25, 8)
    se = math.hypot(coll_ref.std(ddof=1), cont_rej.std(ddof=1)) / math.sqrt(len(coll_ref))
    assert abs(cont_rej.mean() - coll_ref.mean()) < 4.0 * se + 0.02, (cont_rej.mean(), coll_ref.mean(), se)
    assert coll_ref.mean() - coll_rej.mean() > 10.0 * se
