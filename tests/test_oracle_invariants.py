"""Invariants and special cases of the oracle's sweep (Sec. 3.4)."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import ecmc_workloads as W
import oracle


def small_params(**kw):
    w = W.SMALL
    p = dict(N=w.N, L=w.L, sigma=1.0, cells_x=2, cells_y=2, ell=4.0, n_m=2, seed=1)
    p.update(kw)
    return oracle.make_params(**p)


def run(p, n, t0=0, x=None, y=None):
    if x is None:
        x, y = W.square_lattice(p.N, p.L)
    x, y = x.copy(), y.copy()
    st, recs = oracle.sweeps(p, x, y, t0, n, records=True)
    return x, y, st, recs


# -- (a) no overlap ---------------------------------------------------------
@pytest.mark.parametrize("N,eta,cells,ell,nm", [
    (256, 0.70, 2, 4.0, 2), (1024, 0.72, 4, 8.0, 2), (1024, 0.72, 8, 2.0, 1),
    (4096, 0.72, 16, 8.0, 1), (576, 0.75, 6, 3.0, 3)])
def test_no_overlap(N, eta, cells, ell, nm):
    L = W.box_side(N, eta)
    p = oracle.make_params(N, L, 1.0, cells, cells, ell, nm, 3)
    x, y = W.square_lattice(N, L)
    for _ in range(5):
        oracle.sweeps(p, x, y, 0, 10)
        assert oracle.min_dist2(L, x, y) >= 1.0 - 1e-12
        assert np.all((x >= 0) & (x < L) & (y >= 0) & (y < L))


# -- cells of one colour are independent (checkerboard, Sec. 3.4) -----------
def test_cell_order_within_colour_is_irrelevant():
    N, eta = 1024, 0.72
    L = W.box_side(N, eta)
    a = run(oracle.make_params(N, L, 1.0, 8, 8, 4.0, 2, 5), 10)
    b = run(oracle.make_params(N, L, 1.0, 8, 8, 4.0, 2, 5, flags=oracle.FLAG_REVERSE_CELLS), 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[2].events == b[2].events and np.array_equal(a[3], b[3])


def test_neighbour_cells_hold_every_frozen_image():
    # frozen sets from the 3x3 block of cells equal those from all disks
    for cells in (2, 4):
        N, eta = 256, 0.70
        L = W.box_side(N, eta)
        a = run(oracle.make_params(N, L, 1.0, cells, cells, 4.0, 2, 9), 8)
        b = run(oracle.make_params(N, L, 1.0, cells, cells, 4.0, 2, 9,
                                   flags=oracle.FLAG_BRUTE_FROZEN), 8)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_single_start_lists_coincide():
    # with n_m = 1 the two list rules give the same sweep (Sec. 3.4)
    a = run(small_params(n_m=1), 10)
    b = run(small_params(n_m=1, list_mode=oracle.LIST_WITHOUT_REPL), 10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = run(small_params(n_m=3), 3)
    d = run(small_params(n_m=3, list_mode=oracle.LIST_WITHOUT_REPL), 3)
    assert not np.array_equal(c[0], d[0])


def test_without_replacement_starts_are_distinct():
    p = small_params(n_m=20, list_mode=oracle.LIST_WITHOUT_REPL)
    _, _, _, recs = run(p, 3)
    for s in range(3):
        for c in range(4):
            starts = recs[s, c]["start_id"]
            # all distinct while n_m <= n_c (here n_c ~ 64)
            assert len(set(starts.tolist())) == len(starts)


def test_with_replacement_starts_repeat():
    p = small_params(n_m=40)
    _, _, _, recs = run(p, 20)
    rep = sum(len(set(recs[s, c]["start_id"].tolist())) < 40 for s in range(20) for c in range(4))
    assert rep > 40  # birthday collisions are the rule at 40 draws from ~64


def test_chain_records_are_consistent():
    p = small_params()
    x, y, st, recs = run(p, 20)
    assert st.chains == 20 * 4 * 2
    assert recs["events"].sum() == st.events and recs["walls"].sum() == st.wall_hits
    assert st.lifts + st.frozen_hits == st.events
    assert st.sum_disp == pytest.approx(st.chains * 4.0)


def test_resume_is_bitwise_identical():
    p = small_params()
    a = run(p, 10)
    x, y, _, _ = run(p, 4)
    x2, y2 = x.copy(), y.copy()
    oracle.sweeps(p, x2, y2, 4, 6)
    assert np.array_equal(a[0], x2) and np.array_equal(a[1], y2)


def test_zero_displacement_is_identity_up_to_frame_rounding():
    p = small_params(ell=0.0)
    x0, y0 = W.square_lattice(p.N, p.L)
    x, y, st, _ = run(p, 5)
    assert st.events == 0 and np.max(np.abs(x - x0)) < 1e-12 and np.max(np.abs(y - y0)) < 1e-12


def test_default_chains_per_cell_eq_nm():
    # eq. (nm) with lambda0 = sigma (eta_hcp - eta) / (2 eta_hcp)
    for N, eta, cells, ell, expect in [(256, 0.70, 2, 4.0, 2), (65536, 0.708, 32, 8.0, 1),
                                       (1048576, 0.72, 128, 8.0, 1),
                                       (1048576, 0.72, 8, 2.0, 844)]:
        L = W.box_side(N, eta)
        lam = (W.ETA_HCP - eta) / (2 * W.ETA_HCP)
        direct = max(1, int(math.floor(N / cells**2 * lam / ell + 0.5)))
        assert oracle.default_nm(N, L, 1.0, cells, cells, ell) == direct == expect


# -- per-sweep draws (Sec. 3.4 steps 1-3) ------------------------------------
def test_colour_orders_are_uniform_permutations():
    p = small_params()
    counts = {}
    for t in range(24000):
        sx, sy, perm = oracle.sweep_draws(p, t)
        assert sorted(perm) == [0, 1, 2, 3]
        counts[tuple(perm)] = counts.get(tuple(perm), 0) + 1
    assert set(counts) == set(itertools.permutations(range(4)))
    chi2 = sum((c - 1000.0) ** 2 / 1000.0 for c in counts.values())
    assert chi2 < 60.0  # 23 degrees of freedom


def test_shift_is_uniform_in_cell():
    p = small_params()
    w = p.L / 2
    s = np.array([oracle.sweep_draws(p, t)[:2] for t in range(20000)])
    assert np.all((s >= 0) & (s < w))
    hist = np.histogram(s[:, 0], bins=20, range=(0, w))[0]
    assert np.sum((hist - 1000.0) ** 2 / 1000.0) < 55.0
    assert abs(np.corrcoef(s[:, 0], s[:, 1])[0, 1]) < 0.03


def test_binning_matches_exact_arithmetic():
    N, eta = 4096, 0.72
    L = W.box_side(N, eta)
    p = oracle.make_params(N, L, 1.0, 16, 16, 2.0, 1, 4)
    x, y = W.square_lattice(N, L)
    oracle.sweeps(p, x, y, 0, 3)
    cell = oracle.bin_cells(p, 3, x, y)
    sx, sy, _ = oracle.sweep_draws(p, 3)
    w = Fraction(L) / 16
    bad = 0
    for i in range(0, N, 7):
        for v, s, c in ((x[i], sx, cell[i] % 16), (y[i], sy, cell[i] // 16)):
            u = (Fraction(v) - Fraction(s)) % Fraction(L)
            exact = min(int(u / w), 15)
            if exact != c:
                # only a centre within rounding of a cell wall may differ
                assert abs(float(u - exact * w)) < 1e-12 or abs(float(u - c * w)) < 1e-12
                bad += 1
    assert bad <= 2
    assert np.bincount(cell, minlength=256).sum() == N


# -- 1 disk in a fixed cell: stationarity of the direction rule --------------
def one_disk(x0, dir_mode, t=0):
    L = 10.0
    p = oracle.make_params(1, L, 1.0, 2, 2, 2.5, 1, 17, 0, dir_mode=dir_mode,
                           flags=oracle.FLAG_NO_SHIFT)
    out = []
    for r, xv in enumerate(x0):
        p.replica = r
        x, y = np.array([xv]), np.array([2.5])
        oracle.sweeps(p, x, y, t, 1)
        out.append(x[0])
    return np.array(out)


def test_single_disk_positive_only_folds_into_upper_half():
    # +x only with ell = w/2: x -> x + w/2 below w/2, x -> 3w/2 - x above
    x0 = (np.arange(400) + 0.5) * 5.0 / 400
    x1 = one_disk(x0, oracle.DIR_POS_ONLY)
    expect = np.where(x0 < 2.5, x0 + 2.5, 7.5 - x0)
    assert np.max(np.abs(x1 - expect)) < 1e-12
    assert np.all(x1 >= 2.5)


def test_single_disk_plus_minus_keeps_uniform_density():
    x0 = (np.arange(4000) + 0.5) * 5.0 / 4000
    x1 = one_disk(x0, oracle.DIR_PM_AXIS_ALT)
    plus = np.where(x0 < 2.5, x0 + 2.5, 7.5 - x0)
    minus = np.where(x0 >= 2.5, x0 - 2.5, 2.5 - x0)
    ok = (np.abs(x1 - plus) < 1e-12) | (np.abs(x1 - minus) < 1e-12)
    assert ok.all()
    hist = np.histogram(x1, bins=10, range=(0, 5))[0]
    assert np.sum((hist - 400.0) ** 2 / 400.0) < 30.0  # 9 degrees of freedom


# -- no disk passes through another ------------------------------------------
def cyclic_orders_kept(along0, along1, across, L):
    """Disks less than sigma apart across the axis can never pass each other
    along it, so in every sigma-wide strip across the axis the cyclic order
    along the axis is the same after a sweep as before."""
    strip = np.floor(across).astype(np.int64)
    checked = 0
    for q in np.unique(strip):
        ids = np.flatnonzero(strip == q)
        if len(ids) < 3:
            continue
        before = ids[np.argsort(along0[ids], kind="stable")].tolist()
        after = ids[np.argsort(along1[ids], kind="stable")].tolist()
        k = after.index(before[0])
        if after[k:] + after[:k] != before:
            return False, checked
        checked += 1
    return True, checked


@pytest.mark.parametrize("boundary", [oracle.BOUNDARY_REFLECT, oracle.BOUNDARY_REJECT])
@pytest.mark.parametrize("N,cells,ell,nm", [(4096, 16, 1.5, 6),
                                            (1024, 2, 4.0, 64)])  # frames span half the box
def test_chains_never_carry_a_disk_through_another(boundary, N, cells, ell, nm):
    eta = 0.72
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, cells, cells, ell, nm, 13, boundary=boundary)
    oracle.sweeps(p, x, y, 0, 4)
    for t in range(4, 10):
        x0, y0 = x.copy(), y.copy()
        oracle.sweeps(p, x, y, t, 1)
        along0, along1, across = (x0, x, y0) if t % 2 == 0 else (y0, y, x0)
        ok, checked = cyclic_orders_kept(along0, along1, across, L)
        assert ok, "a disk passed through another in sweep %d" % t
        assert checked >= 0.8 * math.floor(L)  # nearly every strip holds 3 or more
