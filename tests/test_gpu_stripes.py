"""Parity of the CUDA striped decomposition (include/ecmc_stripes.h) with the
oracle's orc_stripe_sweeps, through the C ABI.

Both sides evaluate every contact with the same FP64 expressions (no
contraction), so the stripe of every disk and the chain records are compared
exactly, positions to 1e-12 relative (identical in practice) after every
sweep, the counters exactly and the pressure sums to 1e-11.  Cases: two
stripes (the two neighbours of a stripe coincide and a frozen disk can enter
the band twice), several stripe counts for both boundary rules, a ragged
N = 900, a sparse system with empty stripes, chains much longer than the box
(movers wrap round the periodic axis many times), shuffled start lists, and
the Fig. 3 system N = 256^2 at eta = 0.708 -- each with the sorted-frame
kernel and with the block-wide scan.  Then the low-density pressure of the
reflecting rule against the virial series.
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

from test_oracle_gcontact import virial_golden  # noqa: E402

REL = 1e-12
REJECT, REFLECT = oracle.BOUNDARY_REJECT, oracle.BOUNDARY_REFLECT


def make(N, eta, S, ell, nm, seed, boundary, replica=0, kernel=1, list_mode=0):
    L = W.box_side(N, eta)
    g = P.EcmcStripes(N, L, 1.0, S, ell, seed)
    g.set_param(E.PARAM_STRIPES_N_CHAINS, nm)
    g.set_param(E.PARAM_STRIPES_BOUNDARY, boundary)
    g.set_param(E.PARAM_STRIPES_REPLICA, replica)
    g.set_param(E.PARAM_STRIPES_KERNEL, kernel)
    g.set_param(E.PARAM_STRIPES_LIST_MODE, list_mode)
    assert g.get_param(E.PARAM_STRIPES_KERNEL) == kernel
    p = oracle.make_params(N, L, 1.0, S, S, ell, nm, seed, replica, boundary=boundary,
                           list_mode=list_mode)
    return g, p, L


def interleave(x, y):
    xy = np.empty(2 * x.shape[0])
    xy[0::2], xy[1::2] = x, y
    return xy


def assert_positions_equal(g, x, y, L):
    xy = g.positions()
    worst = 0.0
    for a, ref in enumerate((x, y)):
        d = np.abs(xy[a::2] - ref)
        d = np.minimum(d, L - d)
        worst = max(worst, d.max() / L)
    assert worst <= REL, "max relative position difference %g" % worst


def run_pair(N, eta, S, ell, nm, seed, n_sweeps, boundary, replica=0, kernel=1, list_mode=0):
    g, p, L = make(N, eta, S, ell, nm, seed, boundary, replica, kernel, list_mode)
    x, y = W.square_lattice(N, L)
    g.set_positions(interleave(x, y), t0=0)
    tot = oracle.Stats()
    for s in range(n_sweeps):
        stripes = oracle.stripe_bin(p, s, x, y)
        st, recs = oracle.stripe_sweeps(p, x, y, s, 1, stats=tot, records=True)
        g.sweep(1)
        assert np.array_equal(g.last_stripes(), stripes), "stripes differ at sweep %d" % s
        gr = g.chain_records()
        orr = recs[0]
        assert np.array_equal(gr[:, :, 0], orr["start_id"]), "start disks, sweep %d" % s
        assert np.array_equal(gr[:, :, 1], orr["end_id"]), "end disks, sweep %d" % s
        assert np.array_equal(gr[:, :, 2], orr["events"]), "contacts, sweep %d" % s
        assert_positions_equal(g, x, y, L)
    c = g.counters()
    assert c.events == tot.events and c.lifts == tot.lifts and c.frozen_hits == tot.frozen_hits
    assert c.chains == tot.chains and c.rejected_chains == tot.rejected
    assert c.wall_hits == 0 and c.sweeps == n_sweeps
    assert c.sum_b == pytest.approx(tot.sum_b, rel=1e-11, abs=1e-12)
    assert c.sum_disp == pytest.approx(tot.sum_disp, rel=1e-12)
    if tot.sum_disp_w > 0:
        P_gpu, _ = g.pressure()
        P_or = oracle.pressure_from_sums(tot.sum_b_w, tot.sum_disp_w, N, L, 1.0)
        assert P_gpu == pytest.approx(P_or, rel=1e-11)
    assert g.sweep_index() == n_sweeps
    g.close()
    return tot


KERNELS = [1, 0]  # sorted frames in shared memory; block-wide scan


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("boundary", [REJECT, REFLECT])
@pytest.mark.parametrize("N,eta,S,ell,nm,sweeps", [
    (256, 0.70, 2, 4.0, 4, 10),      # two stripes: both neighbours are one stripe
    (1024, 0.70, 8, 1.3, 8, 10),
    (900, 0.65, 6, 2.0, 5, 8),       # ragged member counts
    (4096, 0.72, 16, 2.0, 3, 6),
])
def test_sweeps_match_oracle(N, eta, S, ell, nm, sweeps, boundary, kernel):
    st = run_pair(N, eta, S, ell, nm, 5, sweeps, boundary, kernel=kernel)
    assert st.events > 0 and st.lifts > 0 and st.frozen_hits > 0
    if boundary == REJECT:
        assert 0 < st.rejected < st.chains


@pytest.mark.parametrize("kernel", KERNELS)
def test_sparse_system_with_empty_stripes(kernel):
    st = run_pair(64, 0.05, 16, 3.0, 2, 3, 12, REJECT, kernel=kernel)
    assert st.chains < 12 * 16 * 2


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("N,eta,S,ell,nm,boundary", [
    (256, 0.30, 4, 60.0, 3, REFLECT),   # L = 25.9: a chain goes round the box twice
    (144, 0.10, 2, 90.0, 4, REFLECT),   # L = 33.6, few contacts, long free flights
    (1024, 0.55, 8, 40.0, 2, REFLECT),
    (256, 0.30, 4, 60.0, 6, REJECT),
])
def test_chains_longer_than_the_box(N, eta, S, ell, nm, boundary, kernel):
    # movers wrap round the periodic axis again and again: the sorted kernel's
    # strips must follow their rotation
    st = run_pair(N, eta, S, ell, nm, 9, 6, boundary, kernel=kernel)
    assert st.events > 0


@pytest.mark.parametrize("boundary", [REJECT, REFLECT])
@pytest.mark.parametrize("N,eta,S,ell,nm", [
    (1024, 0.70, 8, 1.3, 40),           # n_m beyond the members of a stripe: cycled
    (900, 0.65, 6, 2.0, 7),
])
def test_shuffled_start_lists_match_oracle(N, eta, S, ell, nm, boundary):
    st = run_pair(N, eta, S, ell, nm, 21, 4, boundary, list_mode=oracle.LIST_WITHOUT_REPL)
    assert st.events > 0


def test_shuffled_lists_need_the_sorted_kernel():
    g, p, L = make(256, 0.7, 2, 4.0, 2, 1, REJECT, kernel=0)
    g.set_param(E.PARAM_STRIPES_LIST_MODE, oracle.LIST_WITHOUT_REPL)
    with pytest.raises(E.EcmcError) as ei:
        g.sweep(1)
    assert ei.value.code == E.ERR_UNSUPPORTED
    g.close()


@pytest.mark.parametrize("kernel", KERNELS)
def test_fig3_system_two_sweeps(kernel):
    # N = 256^2 at eta = 0.708, stripes of about 8.4 sigma; the sorted frame
    # fits in shared memory, so it is the default there
    g, _, _ = make(65536, 0.708, 32, 8.0, 4, 7, REJECT)
    assert g.get_param(E.PARAM_STRIPES_KERNEL) == 1
    g.close()
    run_pair(65536, 0.708, 32, 8.0, 4, 7, 2, REJECT, kernel=kernel)


def test_replica_key_changes_the_stream():
    a = run_pair(1024, 0.7, 8, 1.3, 4, 5, 2, REFLECT, replica=0)
    b = run_pair(1024, 0.7, 8, 1.3, 4, 5, 2, REFLECT, replica=3)
    assert a.sum_b != b.sum_b


def test_resume_from_positions_is_bitwise():
    g, p, L = make(1024, 0.7, 8, 1.3, 4, 11, REJECT)
    g.sweep(6)
    ref = g.positions().copy()
    g.close()
    g, p, L = make(1024, 0.7, 8, 1.3, 4, 11, REJECT)
    g.sweep(3)
    mid = g.positions().copy()
    g.close()
    g, p, L = make(1024, 0.7, 8, 1.3, 4, 11, REJECT)
    g.set_positions(mid, t0=3)
    g.sweep(3)
    assert np.array_equal(g.positions(), ref)
    g.close()


def test_device_positions_and_caller_stream():
    g, p, L = make(1024, 0.7, 8, 1.3, 4, 13, REFLECT)
    x, y = W.square_lattice(1024, L)
    s = torch.cuda.Stream()
    g.set_stream(s)
    dev = torch.from_numpy(interleave(x, y)).cuda()
    g.set_positions(dev, t0=0)
    g.sweep(3)
    out = torch.empty_like(dev)
    g.positions(out)
    torch.cuda.synchronize()
    oracle.stripe_sweeps(p, x, y, 0, 3)
    assert_positions_equal(g, x, y, L)
    assert np.array_equal(out.cpu().numpy(), g.positions())
    g.close()


def test_low_density_pressure_matches_virial_series():
    # the reflecting rule's collision estimator on the GPU's own sampling
    N, eta = 4096, 0.10
    g, p, L = make(N, eta, 16, 2.0, 40, 17, REFLECT)
    g.sweep(200)
    g.reset_stats()
    g.sweep(4000)
    Pb, se = g.pressure()
    rho = N / L**2
    gv = virial_golden()
    x2 = 0.5 * math.pi * rho
    vir = 1.0 + x2 + gv["B3_over_B2sq"] * x2**2 + gv["B4_over_B2cu"] * x2**3
    z, zse = Pb / rho, se / rho
    assert abs(z - vir) < 4.0 * zse + 1e-3, (z, vir, zse)
    g.close()
