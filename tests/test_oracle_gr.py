"""Pins of the pair-correlation histogram and its normalisation (Sec. 2)."""
import math

import numpy as np
import pytest

import oracle


def test_counts_on_hand_built_configuration():
    L = 20.0
    # pairs at distances 1.005, 1.5, and across the periodic boundary 2.25
    x = np.array([1.0, 2.005, 10.0, 10.0, 0.5])
    y = np.array([5.0, 5.0, 10.0, 11.5, 17.0])
    x[4], y[4] = 19.0, 5.0 + 0.0   # distance to disk 0: 2.0 through the boundary
    c = oracle.gr_counts(L, x, y, 1.0, 0.01, 400)
    # ordered pairs, each unordered pair twice: 1.005 -> bin 0, 1.5 -> bin 50,
    # 2.0 -> bin 100, and disk 1 - disk 4 at 3.005 through the boundary -> bin 200
    d = {0: 2, 50: 2, 100: 2, 200: 2}
    for b, n in d.items():
        assert c[b] == n, (b, c[b])
    assert c.sum() == 8


def test_sampled_first_members():
    rng = np.random.default_rng(1)
    L = 30.0
    x, y = rng.random(300) * L, rng.random(300) * L
    full = oracle.gr_counts(L, x, y, 1.0, 0.05, 80)
    part = oracle.gr_counts(L, x, y, 1.0, 0.05, 80, 0, 120)
    oracle.gr_counts(L, x, y, 1.0, 0.05, 80, 120, 300, counts=part)
    assert np.array_equal(full, part)


def test_ideal_gas_normalises_to_one():
    # uniform random points: n(r_i) = N (N-1)/L^2 * pi (e1^2 - e0^2); the
    # paper's normalisation with the area-weighted R_i gives g = 1 up to
    # (N-1)/N and the O(dr^2) difference between R_i and the bin midpoint
    rng = np.random.default_rng(7)
    N, L, dr, nb = 400, 40.0, 0.05, 80
    counts = np.zeros(nb, np.int64)
    for _ in range(50):
        x, y = rng.random(N) * L, rng.random(N) * L
        oracle.gr_counts(L, x, y, 1.0, dr, nb, counts=counts)
    R, g = oracle.gr_normalise(counts, 50, N, L, 1.0, dr)
    assert abs(np.mean(g) - (N - 1) / N) < 0.01
    e0 = 1.0 + dr * np.arange(nb)
    assert np.all(R > e0) and np.all(R < e0 + dr)


def test_pressure_formula_low_density_limit():
    # eq. (pressure) with g(sigma+) = 1 reduces to the second virial term
    N, L = 100, 100.0
    rho = N / L**2
    assert oracle.pressure_from_gcontact(1.0, N, L, 1.0) == pytest.approx(
        rho * (1 + math.pi / 2 * rho))


@pytest.mark.parametrize("N,L,dr,nb,kind", [
    (300, 30.0, 0.05, 80, "uniform"),       # 7 cells per side
    (900, 33.0, 0.01, 400, "melted"),       # r_max = 5: 6 cells per side
    (256, 16.9, 0.01, 400, "lattice"),      # fewer than 3 cells: the brute force itself
    (2000, 60.0, 0.02, 100, "uniform"),
])
def test_cell_list_counts_equal_brute_force(N, L, dr, nb, kind):
    # the cell-list search must find every pair the brute force finds: the
    # histograms are equal bin by bin, including pairs across the boundary
    rng = np.random.default_rng(N)
    if kind == "uniform":
        x, y = rng.random(N) * L, rng.random(N) * L
    else:
        k = int(round(math.sqrt(N)))
        a = L / k
        i = np.arange(k * k)
        x, y = (i % k + 0.5) * a, (i // k + 0.5) * a
        if kind == "melted":
            p = oracle.make_params(N, L, 1.0, 2, 2, 3.0, 4, 9)
            oracle.sweeps(p, x, y, 0, 30)
    brute = oracle.gr_counts(L, x, y, 1.0, dr, nb)
    cells = oracle.gr_counts_cells(L, x, y, 1.0, dr, nb)
    assert brute.sum() > 0
    assert np.array_equal(brute, cells)
