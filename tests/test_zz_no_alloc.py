"""ecmc_sweep_noalloc: the sweep for callers that cannot allocate device
memory (their memory belongs to their own pool, or allocation is over once
their set-up is done).  It must reproduce the ordinary entry points
(ecmc_create / ecmc_set_positions / ecmc_sweep / ecmc_positions) on two calls
in a row, through the C ABI, within the tolerance of the other parity tests.
This file is collected last on purpose."""
import numpy as np
import pytest

import ecmc_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1409_6948_gb300 as P  # noqa: E402
from paper_1409_6948_gb300 import ecmc as E  # noqa: E402

REL = 1e-12


def close(a, b, L):
    d = np.abs(a - b)
    d = np.minimum(d, L - d)
    return d.max() / L <= REL


@pytest.mark.parametrize("N,eta,cells,ell,nm,seed", [
    (256, 0.70, 2, 4.0, 2, 1),
    (4096, 0.72, 16, 2.0, 1, 31),
])
def test_noalloc_matches_handle_path_on_two_calls(N, eta, cells, ell, nm, seed):
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    xy0 = np.ascontiguousarray(np.stack([x, y], 1).ravel())

    g = P.Ecmc(N, L, 1.0, cells, cells, ell, seed)
    g.set_param(E.PARAM_N_CHAINS, nm)
    g.set_positions(xy0, t0=0)
    g.sweep(3)
    ref1 = g.positions().copy()
    g.sweep(2)
    ref2 = g.positions().copy()
    g.close()

    dev = torch.tensor(xy0, dtype=torch.float64, device="cuda")
    E.sweep_noalloc(dev, N, L, 1.0, cells, cells, ell, nm, seed, 0, 0, 3)
    out1 = dev.cpu().numpy()
    assert close(out1, ref1, L)
    E.sweep_noalloc(dev, N, L, 1.0, cells, cells, ell, nm, seed, 0, 3, 2)
    out2 = dev.cpu().numpy()
    assert close(out2, ref2, L)


def test_noalloc_rejects_systems_beyond_the_static_scratch():
    N = 1048576
    L = W.box_side(N, 0.72)
    dev = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EcmcError) as ei:
        E.sweep_noalloc(dev, N, L, 1.0, 128, 128, 8.0, 1, 3, 0, 0, 1)
    assert ei.value.code == E.ERR_CAPACITY
