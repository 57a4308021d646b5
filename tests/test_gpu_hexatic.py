"""The hexatic order parameter on the GPU against the oracle (eq. Psi).

Both sides decide Delaunay neighbours with the same FP64 expressions and sum
Psi_k over the neighbours in ascending disk id, and Psi over the disks in id
order, so neighbour counts, per-disk Psi_k and Psi agree to the last bit.
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


@pytest.mark.parametrize("N,eta,cells,sweeps", [
    (256, 0.70, 2, 0),      # the square lattice start: degenerate Delaunay graph
    (256, 0.70, 2, 20),     # two cells per side
    (1024, 0.70, 8, 15),
    (4096, 0.72, 16, 10),
])
def test_hexatic_matches_oracle_bitwise(N, eta, cells, sweeps):
    L = W.box_side(N, eta)
    g = P.Ecmc(N, L, 1.0, cells, cells, 3.0, 3)
    g.set_param(E.PARAM_N_CHAINS, 2)
    g.sweep(sweeps)
    xy = g.positions()
    x, y = np.ascontiguousarray(xy[0::2]), np.ascontiguousarray(xy[1::2])
    psi, pk, nn, bad = g.hexatic(per_disk=True)
    opsi, opk, onn, obad = oracle.hexatic(L, x, y)
    assert bad == obad == 0
    assert np.array_equal(nn, onn)
    assert np.array_equal(pk, opk)
    assert psi == opsi
    if sweeps:
        assert nn.sum() == 6 * N  # Euler on the torus
    g.close()


def test_hexatic_of_every_replica_of_a_batch():
    reps = [dict(N=1024, eta=0.70, cells_x=8, cells_y=8, ell=3.0, n_m=2, seed=1, replica=0),
            dict(N=576, eta=0.66, cells_x=6, cells_y=6, ell=2.0, n_m=1, seed=2, replica=3)]
    descs = []
    for d in reps:
        e = dict(d)
        e["L"] = W.box_side(d["N"], d["eta"])
        descs.append(e)
    g = P.Ecmc.batch(descs)
    g.sweep(12)
    xy = g.positions()
    psi, pk, nn, bad = g.hexatic(per_disk=True)
    off = 0
    for r, d in enumerate(descs):
        n = d["N"]
        x = np.ascontiguousarray(xy[2 * off: 2 * (off + n): 2])
        y = np.ascontiguousarray(xy[2 * off + 1: 2 * (off + n): 2])
        opsi, opk, onn, obad = oracle.hexatic(d["L"], x, y)
        assert psi[r] == opsi
        assert np.array_equal(nn[off:off + n], onn) and np.array_equal(pk[off:off + n], opk)
        off += n
    assert bad == 0
    g.close()
