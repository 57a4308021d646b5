"""ecmc_sweep_noalloc: the sweep for callers that cannot allocate device
memory (their memory belongs to their own pool, or allocation is over once
their set-up is done).  It must reproduce the ordinary entry points
(ecmc_create / ecmc_set_positions / ecmc_sweep / ecmc_positions) on two calls
in a row, through the C ABI, within the tolerance of the other parity tests,
and the oracle directly; and it must reject overlapping input, as
ecmc_set_positions does, without touching the caller's positions.
This file is collected last on purpose."""
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


def test_noalloc_matches_the_oracle():
    # N = 1024 is a square, but the entry point takes any N: start from a
    # lattice with 24 disks removed (1000 disks, ids renumbered)
    N0, eta, cells, ell, nm, seed, t0, n = 1024, 0.68, 4, 3.0, 3, 17, 5, 4
    L = W.box_side(N0, eta)
    x, y = W.square_lattice(N0, L)
    keep = np.ones(N0, bool)
    keep[np.arange(0, N0, 43)[:24]] = False
    x, y = x[keep].copy(), y[keep].copy()
    N = x.size
    dev = torch.tensor(np.stack([x, y], 1).ravel(), dtype=torch.float64, device="cuda")
    p = oracle.make_params(N, L, 1.0, cells, cells, ell, nm, seed)
    oracle.sweeps(p, x, y, t0, n)  # in place on x, y
    E.sweep_noalloc(dev, N, L, 1.0, cells, cells, ell, nm, seed, 0, t0, n)
    out = dev.cpu().numpy()
    assert close(out[0::2], x, L) and close(out[1::2], y, L)


def test_noalloc_rejects_overlapping_input_and_keeps_the_positions():
    N, eta, cells = 256, 0.60, 2
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    # disk 1 just under sigma from disk 0, along x (the lattice spacing is
    # above 1.1 sigma, so no other pair comes closer)
    x[1] = x[0] + (1.0 - 1e-6)
    y[1] = y[0]
    xy0 = np.ascontiguousarray(np.stack([x, y], 1).ravel())
    dev = torch.tensor(xy0, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EcmcError) as ei:
        E.sweep_noalloc(dev, N, L, 1.0, cells, cells, 2.0, 1, 3, 0, 0, 2)
    assert ei.value.code == E.ERR_OVERLAP
    assert np.array_equal(dev.cpu().numpy(), xy0)
    # the scratch holds no state across calls: a valid system right after works
    x, y = W.square_lattice(N, L)
    good = torch.tensor(np.stack([x, y], 1).ravel(), dtype=torch.float64, device="cuda")
    E.sweep_noalloc(good, N, L, 1.0, cells, cells, 2.0, 1, 3, 0, 0, 1)


def test_noalloc_rejects_systems_beyond_the_static_scratch():
    N = 1048576
    L = W.box_side(N, 0.72)
    dev = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EcmcError) as ei:
        E.sweep_noalloc(dev, N, L, 1.0, 128, 128, 8.0, 1, 3, 0, 0, 1)
    assert ei.value.code == E.ERR_CAPACITY


def test_noalloc_checks_the_tensor_before_the_call():
    dev = torch.zeros(512, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        E.sweep_noalloc(dev, 256, 16.9, 1.0, 2, 2, 4.0, 1, 1, 0, 0, 1)
    with pytest.raises(ValueError):
        E.sweep_noalloc(torch.zeros(100, dtype=torch.float64, device="cuda"), 256, 16.9, 1.0,
                        2, 2, 4.0, 1, 1, 0, 0, 1)
    with pytest.raises(ValueError):
        E.sweep_noalloc(torch.zeros(512, dtype=torch.float64), 256, 16.9, 1.0, 2, 2, 4.0, 1,
                        1, 0, 0, 1)
