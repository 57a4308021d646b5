"""Pair-correlation counts (Sec. 2) of the CUDA library against the oracle,
bin for bin and exactly.

The library screens pairs on fixed-point squared distances and bins them by
an FP32 estimate of (d - sigma) / dr, falling back to the FP64 expression
near a bin edge; the counts must be the oracle's integers in every case:
lattices whose distances fall exactly on bin edges, melted states at several
bin widths and ranges, the medium workload's binning (0.01 sigma to 5 sigma
at N = 65,536), every replica of a batch, and small boxes that take the FP64
scan.
"""
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


def gpu_counts(g, dr, rmax, replica=0):
    g.set_param(E.PARAM_GR_DR, dr)
    g.set_param(E.PARAM_GR_RMAX, rmax)
    g.gr_measure(replica)
    c, nm = g.gr_counts(replica)
    assert nm == 1
    return c


def test_lattice_distances_on_bin_edges():
    # spacing exactly 1.25 sigma in a box of 40 sigma: pair distances 1.25,
    # 2.5, 3.75, 5 fall exactly on edges of 0.25-wide bins, and on every
    # fourth edge of 0.0625-wide ones
    k, a = 32, 1.25
    L = k * a
    i = np.arange(k * k)
    x, y = (i % k + 0.5) * a, (i // k + 0.5) * a
    g = P.Ecmc(k * k, L, 1.0, 8, 8, 2.0, 1)
    g.set_positions(np.stack([x, y], 1).ravel(), t0=0)
    for dr, rmax in ((0.25, 5.0), (0.0625, 4.0), (0.01, 5.0)):
        nb = int(round((rmax - 1.0) / dr))
        want = oracle.gr_counts(L, x, y, 1.0, dr, nb)
        got = gpu_counts(g, dr, rmax)
        assert np.array_equal(got, want), (dr, np.nonzero(got != want))
        g.reset_stats()
    g.close()


@pytest.mark.parametrize("N,eta,cells,dr,rmax,sweeps", [
    (1024, 0.65, 4, 0.02, 3.0, 5),
    (4096, 0.72, 16, 0.005, 4.0, 4),
    (16384, 0.70, 32, 0.01, 5.0, 3),
    (4096, 0.40, 8, 0.05, 9.0, 3),     # 160 bins, R = 2 cells
])
def test_melted_states(N, eta, cells, dr, rmax, sweeps):
    L = W.box_side(N, eta)
    g = P.Ecmc(N, L, 1.0, cells, cells, 2.0, 5)
    g.sweep(sweeps)
    xy = g.positions()
    x, y = xy[0::2].copy(), xy[1::2].copy()
    nb = int(round((rmax - 1.0) / dr))
    want = oracle.gr_counts_cells(L, x, y, 1.0, dr, nb)
    got = gpu_counts(g, dr, rmax)
    assert want.sum() > 0 and np.array_equal(got, want)
    g.close()


def test_medium_workload_binning_every_replica():
    # N = 65,536 at eta = 0.708, 32x32 cells, g(r) in 0.01 sigma bins to 5
    # sigma, three replicas of a batch measured at once
    N, eta = 65536, 0.708
    L = W.box_side(N, eta)
    g = P.Ecmc.batch([dict(N=N, L=L, cells_x=32, ell=8.0, n_m=1, seed=2, replica=r)
                      for r in range(3)])
    g.set_param(E.PARAM_GR_DR, 0.01)
    g.set_param(E.PARAM_GR_RMAX, 5.0)
    g.sweep(3)
    g.gr_measure(-1)
    xy = g.positions()
    for r in range(3):
        x, y = xy[2 * N * r:2 * N * (r + 1):2].copy(), xy[2 * N * r + 1:2 * N * (r + 1):2].copy()
        want = oracle.gr_counts_cells(L, x, y, 1.0, 0.01, 400)
        got, nm = g.gr_counts(r)
        assert nm == 1 and np.array_equal(got, want), r
    g.close()


def test_small_box_takes_the_fp64_scan():
    # 5 sigma exceeds L/4 in the N = 256 box: the FP64 scan gives the counts
    N, eta = 256, 0.70
    L = W.box_side(N, eta)
    g = P.Ecmc(N, L, 1.0, 2, 2, 4.0, 1)
    g.sweep(3)
    xy = g.positions()
    x, y = xy[0::2].copy(), xy[1::2].copy()
    want = oracle.gr_counts(L, x, y, 1.0, 0.01, 400)
    got = gpu_counts(g, 0.01, 5.0)
    assert np.array_equal(got, want)
    g.close()
