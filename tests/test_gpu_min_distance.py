"""Smallest pair distance (the no-overlap invariant checked by
ecmc_set_positions and returned by ecmc_min_distance) against the oracle's
FP64 minimum, bit for bit.

The CUDA path screens candidates with exact 64-bit integer squared distances
of 32-bit fixed-point positions and evaluates the FP64 formula only for the
candidates an error bound cannot separate; the result must still be the very
double the FP64 formula gives over all pairs.  Cases: jittered lattices up
to N = 2^20 (one unique nearest neighbour per disk), the exact square
lattice (four-way ties everywhere: the rescan path), planted near-ties a few
ulps apart, pairs across the periodic boundary, boxes without pairs inside
2 sigma, few cells per side (the full-neighbourhood variant) and boxes below
8 sigma (the FP64 scan).
"""
import math

import numpy as np
import pytest

import ecmc_workloads as W
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1409_6948_gb300 as P  # noqa: E402
from paper_1409_6948_gb300 import ecmc as E  # noqa: E402


def interleave(x, y):
    xy = np.empty(2 * x.size)
    xy[0::2], xy[1::2] = x, y
    return xy


def jittered_lattice(N, eta, seed, frac=0.98):
    """Square lattice with every coordinate moved by up to frac (a - sigma)/2:
    no two disks overlap and no distances tie."""
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    a = L / int(round(math.sqrt(N)))
    amp = 0.5 * (a - 1.0) * frac
    rng = np.random.default_rng(seed)
    x = np.mod(x + rng.uniform(-amp, amp, N), L)
    y = np.mod(y + rng.uniform(-amp, amp, N), L)
    return L, np.ascontiguousarray(x), np.ascontiguousarray(y)


def gpu_min_distance(N, L, x, y, cells_x, cells_y, seed=1):
    with P.Ecmc(N, L, 1.0, cells_x, cells_y, 2.0, seed) as g:
        g.set_positions(interleave(x, y))
        return g.min_distance()


@pytest.mark.parametrize("N,eta,cx,cy,seed", [
    (4096, 0.70, 8, 8, 1),
    (4096, 0.70, 4, 4, 2),        # four cells per side, R = 1
    (4096, 0.70, 40, 40, 8),      # cells narrower than 2 sigma: R = 2
    (1024, 0.70, 2, 2, 3),        # every cell is a neighbour: full variant
    (4096, 0.70, 16, 2, 4),       # rectangular cells, full variant in y
    (10000, 0.50, 12, 6, 5),      # ragged member counts
    (65536, 0.72, 60, 60, 6),
    (1048576, 0.72, 240, 240, 7),  # the paper's cells at N = 2^20
])
def test_jittered_lattice_bitwise(N, eta, cx, cy, seed):
    L, x, y = jittered_lattice(N, eta, seed)
    ref = math.sqrt(oracle.min_dist2(L, x, y))
    assert ref < 2.0
    assert gpu_min_distance(N, L, x, y, cx, cy) == ref


@pytest.mark.parametrize("N,eta,c", [(4096, 0.70, 8), (65536, 0.70, 32), (1024, 0.6, 2)])
def test_square_lattice_ties(N, eta, c):
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    ref = math.sqrt(oracle.min_dist2(L, x, y))
    assert gpu_min_distance(N, L, x, y, c, c) == ref


def sparse_lattice(k=32, a=3.0):
    """k x k lattice of spacing a > 2 sigma: no pair inside 2 sigma."""
    N, L = k * k, k * a
    x, y = W.square_lattice(N, L)
    return N, L, x.copy(), y.copy()


def test_no_pair_inside_two_sigma_returns_two_sigma():
    N, L, x, y = sparse_lattice()
    assert oracle.min_dist2(L, x, y) == 4.0
    assert gpu_min_distance(N, L, x, y, 8, 8) == 2.0


@pytest.mark.parametrize("seed", range(6))
def test_planted_near_ties(seed):
    # disk 0's right and upper neighbours at 1.5 plus a few ulps each, and a
    # third pair elsewhere: the integer screen cannot order them, FP64 must
    N, L, x, y = sparse_lattice()
    rng = np.random.default_rng(100 + seed)
    k = 32
    base = 1.5
    eps = np.ldexp(1.0, -52)
    i0 = 5 * k + 5
    d = base * (1.0 + eps * rng.integers(-4, 5, 3))
    x[i0 + 1] = x[i0] + d[0]              # right neighbour
    y[i0 + k] = y[i0] + d[1]              # upper neighbour
    j0 = 20 * k + 17
    x[j0 + 1] = x[j0] + d[2]
    ref = math.sqrt(oracle.min_dist2(L, x, y))
    assert ref < 1.6
    for c in (8, 2):
        assert gpu_min_distance(N, L, x, y, c, c) == ref


def test_pair_across_the_periodic_boundary():
    N, L, x, y = sparse_lattice()
    k = 32
    # disk 0 at the left edge; its left neighbour across the boundary
    x[0] = 0.3
    x[k - 1] = L - 0.8 + 1e-13
    ref = math.sqrt(oracle.min_dist2(L, x, y))
    assert abs(ref - 1.1) < 1e-9
    assert gpu_min_distance(N, L, x, y, 8, 8) == ref


def test_touching_pair_is_accepted_and_exact():
    N, L, x, y = sparse_lattice()
    x[1] = x[0] + 1.0
    assert gpu_min_distance(N, L, x, y, 8, 8) == 1.0


@pytest.mark.parametrize("gap", [0.5, 0.0])
def test_overlap_is_rejected(gap):
    N, L, x, y = sparse_lattice()
    x[3], y[3] = x[2] + gap, y[2]  # an overlapping or a coincident pair
    with P.Ecmc(N, L, 1.0, 8, 8, 2.0, 1) as g:
        with pytest.raises(E.EcmcError) as ei:
            g.set_positions(interleave(x, y))
        assert ei.value.code == E.ERR_OVERLAP


@pytest.mark.parametrize("N,eta", [(16, 0.35), (36, 0.6)])
def test_small_box_takes_the_fp64_scan(N, eta):
    # L below 8 sigma: the fixed-point path needs 2 sigma < L / 4
    L, x, y = jittered_lattice(N, eta, 9)
    assert L < 8.0
    ref = math.sqrt(oracle.min_dist2(L, x, y))
    assert gpu_min_distance(N, L, x, y, 2, 2) == ref
