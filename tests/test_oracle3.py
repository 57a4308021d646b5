"""Pins of the three-dimensional oracle (hard spheres; the generalisation of
the sweep of Sec. 3.4 to cubic cells in 2x2x2 blocks).

  - closed forms of single chains on hand-built frames: head-on lift, an
    offset contact with the impact parameter split over both perpendicular
    axes (s = b - sqrt(sigma^2 - c^2)), every axis and sign, spheres beside
    and behind, a frozen sphere and a wall turning the chain back, ties;
  - one sphere per cell with no contact possible: the chain's end is the
    fold of x +- ell into [0, w], recomputed from Philox;
  - the pressure against the virial series (B2 = 2 pi sigma^3 / 3, B3 and B4
    from tests/golden/hard_sphere_virial.txt, itself checked against the
    closed forms) at eta = 0.05 and the Carnahan-Starling equation at
    eta = 0.3;
  - no overlap after dense sweeps; identical trajectories when the cells of
    a colour are visited in reverse or the frozen set is taken from all
    spheres; the colour order is a permutation of the eight colours;
  - three spheres in a periodic cube: the sampled pair-distance histogram
    below L/2 matches the exact distribution of the uniform measure
    (tests/threesphere_exact.py, itself checked against rejection sampling).
    A sign always + or a chain that stops at the wall instead of turning
    back fails it by orders of magnitude.
"""
import math

import numpy as np
import pytest

import ecmc_workloads as W
import oracle
import threesphere_exact as T3

W_CELL = 10.0


def chain(X, Y, Z, n_mem, m, axis, sign, ell, imgs=None, ids=None):
    return oracle.run_chain_frame3(X, Y, Z, n_mem, m, axis, sign, ell, W_CELL, imgs=imgs,
                                   ids=ids)


def test_head_on_lift_along_z():
    X, Y, Z, st, rec = chain([5, 5], [5, 5], [1.0, 3.5], 2, 0, 2, 1, 2.0)
    assert Z.tolist() == [2.5, 4.0] and X.tolist() == [5, 5] and Y.tolist() == [5, 5]
    assert st.events == 1 and st.lifts == 1 and rec["end_id"] == 1
    assert st.sum_b == pytest.approx(1.0, abs=1e-15)


def test_offset_contact_over_both_perpendicular_axes():
    # c^2 = 0.36^2 + 0.48^2 = 0.36: contact after b - sqrt(1 - 0.36) = 3 - 0.8
    X, Y, Z, st, rec = chain([5.0, 5.36], [5.0, 5.48], [1.0, 4.0], 2, 0, 2, 1, 3.0)
    assert Z[0] == pytest.approx(3.2, abs=1e-14) and Z[1] == pytest.approx(4.8, abs=1e-14)
    assert st.sum_b == pytest.approx(0.8, abs=1e-14)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("sign", [1, -1])
def test_every_axis_and_sign(axis, sign):
    A = [5.0, 5.0, 5.0]
    B = [5.0, 5.0, 5.0]
    B[axis] += sign * 2.5
    C = [list(v) for v in zip(A, B)]
    X, Y, Z, st, _ = chain(C[0], C[1], C[2], 2, 0, axis, sign, 2.0)
    out = [X, Y, Z]
    assert out[axis][0] == 5.0 + sign * 1.5 and out[axis][1] == 5.0 + sign * 3.0
    assert st.lifts == 1


def test_beside_and_behind_are_not_hit():
    # sphere 1 beside (c = sigma exactly: no hit), sphere 2 behind
    X, Y, Z, st, _ = chain([5, 6, 5], [5, 5, 5], [2, 4, 1.5], 3, 0, 2, 1, 2.0)
    assert Z.tolist() == [4.0, 4.0, 1.5] and st.events == 0


def test_frozen_sphere_turns_the_chain_back():
    # member at z = 3, frozen sphere at z = 5.5: contact after 1.5, back 1.0
    X, Y, Z, st, _ = chain([5, 5], [5, 5], [3.0, 5.5], 1, 0, 2, 1, 2.5)
    assert Z[0] == 3.5 and st.frozen_hits == 1 and st.events == 1
    assert st.sum_b == pytest.approx(1.0, abs=1e-15)


def test_wall_turns_the_chain_back():
    X, Y, Z, st, _ = chain([8.5], [5.0], [5.0], 1, 0, 0, 1, 4.0)
    assert X[0] == 10.0 - 2.5 and st.wall_hits == 1 and st.events == 0


def test_equal_distance_tie_takes_smaller_key():
    # two members at the same hit distance (offsets +-0.25 in x): the one
    # with the smaller key (id 3) is lifted and carries the rest of the budget
    X, Y, Z, st, rec = chain([5, 5.25, 4.75], [5, 5, 5], [2, 4, 4], 3, 0, 2, 1, 1.5,
                             ids=[0, 5, 3])
    assert st.lifts == 1 and rec["end_id"] == 3
    assert Z[1] == 4.0 and Z[2] > 4.0


def fold(u, w):
    u = u % (2 * w)
    return 2 * w - u if u > w else u


@pytest.mark.parametrize("seed", range(6))
def test_one_sphere_per_cell_folds(seed):
    # 2x2x2 cells of side 5 without shift; sweep 0 runs along x.  Spheres
    # of x-neighbouring cells differ by 2 in y, so no contact is possible
    L, ell = 10.0, 7.3
    rng = np.random.default_rng(seed)
    x, y, z = [], [], []
    cells = []
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                x.append(5.0 * cx + rng.uniform(0.2, 4.8))
                y.append(5.0 * cy + 0.5 + 2.0 * cx + rng.uniform(0, 0.5))
                z.append(5.0 * cz + 2.5)
                cells.append((cz * 2 + cy) * 2 + cx)
    x, y, z = np.array(x), np.array(y), np.array(z)
    p = oracle.make_params3(8, L, 1.0, 2, ell, 1, 50 + seed, flags=oracle.FLAG_NO_SHIFT)
    xe = x.copy()
    for i in range(8):
        v = oracle.philox([0, 1, cells[i], 0], [50 + seed, 0])
        sg = -1.0 if (v[1] >> 63) else 1.0
        cx = int(x[i] // 5.0)
        xe[i] = 5.0 * cx + fold(x[i] - 5.0 * cx + sg * ell, 5.0)
    xx, yy, zz = x.copy(), y.copy(), z.copy()
    st, _ = oracle.sweeps3(p, xx, yy, zz, 0, 1)
    assert st.events == 0 and st.chains == 8
    np.testing.assert_allclose(xx, xe, rtol=0, atol=1e-12)
    assert yy.tolist() == y.tolist() and zz.tolist() == z.tolist()


def pressure_batches(N, eta, cells, ell, nm, melt, nbatch, per_batch, seed):
    L = W.box_side3(N, eta)
    x, y, z = W.cubic_lattice(N, L)
    p = oracle.make_params3(N, L, 1.0, cells, ell, nm, seed)
    oracle.sweeps3(p, x, y, z, 0, melt)
    vals = []
    t = melt
    for _ in range(nbatch):
        st, _ = oracle.sweeps3(p, x, y, z, t, per_batch)
        t += per_batch
        vals.append(st.sum_b_w / st.sum_disp_w)  # beta P / rho - 1
    vals = np.array(vals)
    return 1.0 + vals.mean(), vals.std(ddof=1) / math.sqrt(nbatch), L


def sphere_virial_golden():
    import os

    here = os.path.dirname(os.path.abspath(__file__))
    vals = {}
    with open(os.path.join(here, "golden", "hard_sphere_virial.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_sphere_virial_golden_matches_closed_forms():
    v = sphere_virial_golden()
    assert v["B3_over_B2sq"] == 0.625
    b4 = (2707 * math.pi + 438 * math.sqrt(2.0) - 4131 * math.acos(1.0 / 3.0)) / (4480 * math.pi)
    assert abs(v["B4_over_B2cu"] - b4) < 1e-10


def test_low_density_pressure_matches_virial_series():
    N, eta = 1000, 0.05
    z, se, L = pressure_batches(N, eta, 4, 3.0, 20, 20, 20, 40, 3)
    v = sphere_virial_golden()
    B2 = 2.0 * math.pi / 3.0
    rho = N / L**3
    x = B2 * rho
    virial = 1.0 + x + v["B3_over_B2sq"] * x**2 + v["B4_over_B2cu"] * x**3
    assert abs(z - virial) < 3.5 * se + 1e-3, (z, virial, se)


def test_moderate_density_pressure_matches_carnahan_starling():
    N, eta = 512, 0.30
    z, se, L = pressure_batches(N, eta, 2, 2.0, 30, 50, 20, 25, 4)
    cs = (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3
    assert abs(z - cs) < 3.5 * se + 0.004 * cs, (z, cs, se)


def test_dense_sweeps_keep_spheres_apart():
    N, eta = 512, 0.50
    L = W.box_side3(N, eta)
    x, y, z = W.cubic_lattice(N, L)
    p = oracle.make_params3(N, L, 1.0, 2, 1.0, 20, 5)
    st, _ = oracle.sweeps3(p, x, y, z, 0, 30)
    assert st.events > 10000 and st.frozen_hits > 0 and st.wall_hits > 0
    assert oracle.min_dist2_3(L, x, y, z) >= 1.0 - 1e-12


@pytest.mark.parametrize("flag", [oracle.FLAG_REVERSE_CELLS, oracle.FLAG_BRUTE_FROZEN])
def test_cell_order_and_frozen_set_do_not_change_the_trajectory(flag):
    N, eta = 216, 0.45
    L = W.box_side3(N, eta)
    a = W.cubic_lattice(N, L)
    b = [v.copy() for v in a]
    a = [v.copy() for v in a]
    p = oracle.make_params3(N, L, 1.0, 2, 1.5, 6, 9)
    q = oracle.make_params3(N, L, 1.0, 2, 1.5, 6, 9, flags=flag)
    sa, _ = oracle.sweeps3(p, *a, 0, 8)
    sb, _ = oracle.sweeps3(q, *b, 0, 8)
    for u, v in zip(a, b):
        assert u.tolist() == v.tolist()
    assert sa.events == sb.events and sa.sum_b == sb.sum_b


def test_colour_orders_are_permutations():
    p = oracle.make_params3(8, 10.0, 1.0, 2, 1.0, 1, 3)
    seen = set()
    for t in range(200):
        sh, perm = oracle.sweep_draws3(p, t)
        assert sorted(perm) == list(range(8))
        assert all(0.0 <= s < 5.0 for s in sh)
        seen.add(tuple(perm))
    assert len(seen) > 190  # 8! orders: repeats are rare


# -- three spheres: the uniform measure ----------------------------------------
L3S = 3.2
EDGES3 = np.linspace(1.0, 0.5 * L3S, 11)


def test_exact_three_sphere_distribution_matches_rejection_sampling():
    p = T3.bin_probabilities(EDGES3, L3S, 1.0)
    assert np.abs(T3.bin_probabilities(EDGES3, L3S, 1.0, n_dir=12000, n_r=20) / p - 1).max() < 1e-7
    rng = np.random.default_rng(5)
    hist = np.zeros(len(EDGES3) - 1)
    for _ in range(8):
        P = rng.random((500_000, 3, 3)) * L3S

        def md(a, b):
            d = a - b
            d -= L3S * np.round(d / L3S)
            return np.sqrt((d * d).sum(-1))

        d12, d13, d23 = md(P[:, 0], P[:, 1]), md(P[:, 0], P[:, 2]), md(P[:, 1], P[:, 2])
        ok = (d12 >= 1.0) & (d13 >= 1.0) & (d23 >= 1.0)
        hist += np.histogram(np.concatenate([d12[ok], d13[ok], d23[ok]]), EDGES3)[0]
    n = hist.sum() / 3.0  # conservative: the three pairs of a sample are dependent
    z = (hist / hist.sum() - p) / np.sqrt(p * (1 - p) / n)
    assert np.max(np.abs(z)) < 5.0


@pytest.mark.parametrize("ell,nm", [(2.0, 4), (0.7, 2)])
def test_three_spheres_sample_the_uniform_measure(ell, nm):
    x = np.array([0.3, 1.5, 2.6])
    y = np.array([0.4, 2.1, 1.1])
    z = np.array([0.2, 1.2, 2.5])
    p3 = oracle.make_params3(3, L3S, 1.0, 2, ell, nm, 3)
    oracle.sweeps3(p3, x, y, z, 0, 100)
    n = 200_000
    S = np.empty((n, 3, 3))
    st = oracle.Stats()
    for s in range(n):
        oracle.sweeps3(p3, x, y, z, 100 + s, 1, stats=st)
        S[s, :, 0], S[s, :, 1], S[s, :, 2] = x, y, z

    def md(i, j):
        d = S[:, i] - S[:, j]
        d -= L3S * np.round(d / L3S)
        return np.sqrt((d * d).sum(-1))

    d = np.stack([md(0, 1), md(0, 2), md(1, 2)], 1)
    hb = np.array([np.histogram(b.ravel(), EDGES3)[0] for b in np.array_split(d, 50)], float)
    hb /= hb.sum(1, keepdims=True)
    se = hb.std(0, ddof=1) / math.sqrt(50)
    zz = (hb.mean(0) - T3.bin_probabilities(EDGES3, L3S, 1.0)) / se
    assert st.frozen_hits > 0 and st.wall_hits > 0 and st.lifts > 0
    assert np.mean(zz**2) < 2.5 and np.max(np.abs(zz)) < 4.5


def test_chains_never_carry_a_sphere_through_another():
    # spheres in one column of side sigma / sqrt 2 across the axis are less
    # than sigma apart across it, so they can never pass each other along
    # it: the cyclic order along the axis in every column survives a sweep
    N, eta = 4096, 0.45
    L = W.box_side3(N, eta)
    x, y, z = W.cubic_lattice(N, L)
    p = oracle.make_params3(N, L, 1.0, 8, 2.0, 4, 17)
    oracle.sweeps3(p, x, y, z, 0, 3)
    side = 1.0 / math.sqrt(2.0)
    checked = 0
    for t in range(3, 9):
        before = [x.copy(), y.copy(), z.copy()]
        oracle.sweeps3(p, x, y, z, t, 1)
        a = t % 3
        pa, qa = [k for k in range(3) if k != a]
        col = (np.floor(before[pa] / side).astype(np.int64) * 100000
               + np.floor(before[qa] / side).astype(np.int64))
        after = [x, y, z][a]
        for c in np.unique(col):
            ids = np.flatnonzero(col == c)
            if len(ids) < 3:
                continue
            o0 = ids[np.argsort(before[a][ids], kind="stable")].tolist()
            o1 = ids[np.argsort(after[ids], kind="stable")].tolist()
            k = o1.index(o0[0])
            assert o1[k:] + o1[:k] == o0, "a sphere passed through another in sweep %d" % t
            checked += 1
        # across the axis only the frame round trip's rounding moves a sphere
        assert np.abs(before[pa] - [x, y, z][pa]).max() < 1e-12 * L
    assert checked > 100
