"""Pins of the oracle's hexatic order parameter (Sec. 2, eq. Psi).

Next neighbours are the Delaunay neighbours (the paper triangulates with a
library); the oracle decides them by clipping bisectors.  Pinned by:
  - a triangular patch: interior disks have 6 neighbours at multiples of 60
    degrees, so Psi_k = 1;
  - Euler's formula on the torus: a periodic Delaunay triangulation has
    exactly 3N edges, so the neighbour counts sum to 6N;
  - scipy's Delaunay triangulation of the 3x3 periodic tiling: the same
    neighbour set for every disk;
  - a rotation of the box by 90 degrees multiplies every exp(6 i phi) by
    exp(6 i pi/2) = -1.
"""
import math

import numpy as np
import pytest

import ecmc_workloads as W
import oracle


def gas(N, eta, seed):
    """A disordered configuration: the square lattice melted by 30 sweeps of
    the oracle (a random configuration without degeneracies)."""
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    cells = max(2, 2 * int(L / 4.0 / 2))
    p = oracle.make_params(N, L, 1.0, cells, cells, 2.0, 4, seed)
    oracle.sweeps(p, x, y, 0, 30)
    return L, np.ascontiguousarray(x), np.ascontiguousarray(y)


def test_triangular_patch_interior_is_perfectly_ordered():
    a = 1.1
    rows, cols = 16, 16
    xs, ys = [], []
    for r in range(rows):
        for c in range(cols):
            xs.append(20.0 + c * a + (0.5 * a if r % 2 else 0.0))
            ys.append(20.0 + r * a * math.sqrt(3.0) / 2.0)
    x, y = np.array(xs), np.array(ys)
    L = 80.0
    psi, pk, nn, bad = oracle.hexatic(L, x, y, rs=3.5)
    interior = [(r * cols + c) for r in range(3, rows - 3) for c in range(3, cols - 3)]
    assert np.all(nn[interior] == 6)
    assert np.allclose(pk[interior], 1.0, atol=1e-12)
    assert bad > 0  # cells of the patch's rim reach beyond rs/2 and are flagged


@pytest.mark.parametrize("N,eta,seed", [(196, 0.5, 1), (400, 0.65, 2), (256, 0.7, 3)])
def test_neighbour_counts_obey_euler(N, eta, seed):
    L, x, y = gas(N, eta, seed)
    psi, pk, nn, bad = oracle.hexatic(L, x, y, rs=min(3.5, 0.49 * L))
    assert bad == 0
    assert nn.sum() == 6 * N


def periodic_delaunay_neighbours(L, x, y):
    spatial = pytest.importorskip("scipy.spatial")
    N = x.size
    pts, idx = [], []
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            pts.append(np.stack([x + sx * L, y + sy * L], 1))
            idx.append(np.arange(N))
    pts = np.concatenate(pts)
    idx = np.concatenate(idx)
    tri = spatial.Delaunay(pts)
    nb = [set() for _ in range(N)]
    central = np.arange(4 * N, 5 * N)  # the (0, 0) copy
    cset = set(central.tolist())
    for simplex in tri.simplices:
        for i in simplex:
            if i in cset:
                for j in simplex:
                    if j != i:
                        nb[i - 4 * N].add(int(j))
    return nb, pts


@pytest.mark.parametrize("N,eta,seed", [(144, 0.5, 4), (324, 0.68, 5)])
def test_neighbours_match_scipy_delaunay(N, eta, seed):
    L, x, y = gas(N, eta, seed)
    nb, pts = periodic_delaunay_neighbours(L, x, y)
    psi, pk, nn, bad = oracle.hexatic(L, x, y, rs=min(3.5, 0.49 * L))
    assert bad == 0
    assert [len(s) for s in nb] == nn.tolist()
    # Psi_k from scipy's neighbour sets, in numpy
    ref = np.empty(N, complex)
    for k in range(N):
        d = np.array([pts[j] - pts[4 * N + k] for j in nb[k]])
        z = d[:, 0] + 1j * d[:, 1]
        ref[k] = np.mean((z / np.abs(z)) ** 6)
    assert np.allclose(pk, ref, atol=1e-12)
    assert abs(psi - ref.mean()) < 1e-12


def test_rotation_by_a_right_angle_flips_psi():
    N, eta = 400, 0.7
    L, x, y = gas(N, eta, 6)
    psi, _, nn, bad = oracle.hexatic(L, x, y)
    xr = np.ascontiguousarray(np.mod(-y, L))
    yr = np.ascontiguousarray(x.copy())
    psi_r, _, nn_r, bad_r = oracle.hexatic(L, xr, yr)
    assert bad == 0 and bad_r == 0
    assert np.array_equal(nn, nn_r)
    assert abs(psi_r + psi) < 1e-12


def test_dense_lattice_start_is_square_symmetric():
    # the square lattice start: Delaunay is degenerate (4 co-circular
    # disks), the diagonal bisectors shrink to points and are no edges; the 4
    # axis neighbours contribute exp(6 i k pi/2) = (-1)^k, so Psi = 0
    N, eta = 256, 0.7
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    psi, pk, nn, bad = oracle.hexatic(L, x, y)
    assert np.all(nn == 4)
    assert abs(psi) < 1e-12
