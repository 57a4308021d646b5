"""Parity of the three-dimensional CUDA sweep (include/ecmc3.h) with the
oracle's orc3_sweeps, through the C ABI.

Both sides evaluate every contact with the same FP64 expressions (no
contraction), so the binning and the chain records are compared exactly,
positions to 1e-12 relative (identical in practice) after every sweep, the
counters exactly and the pressure to 1e-11.  Cases: two cells per side (the
neighbour cells coincide), several cell counts, a ragged N = 10^3, n_m from 1
to 6, and dense systems with many frozen contacts.  The overlap check and
the smallest distance are compared with the oracle's grid search.
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

REL = 1e-12


def make3(N, eta, cells, ell, nm, seed, persistent=1, replay=1):
    L = W.box_side3(N, eta)
    g = P.Ecmc3(N, L, 1.0, cells, ell, seed)
    g.set_param(E.PARAM3_N_CHAINS, nm)
    g.set_param(E.PARAM3_PERSISTENT, persistent)
    g.set_param(E.PARAM3_REPLAY, replay)
    p = oracle.make_params3(N, L, 1.0, cells, ell, nm, seed)
    return g, p, L


def assert_positions_equal(g, x, y, z, L):
    xyz = g.positions()
    worst = 0.0
    for a, ref in enumerate((x, y, z)):
        d = np.abs(xyz[a::3] - ref)
        d = np.minimum(d, L - d)
        worst = max(worst, d.max() / L)
    assert worst <= REL, "max relative position difference %g" % worst


def run_pair3(N, eta, cells, ell, nm, seed, n_sweeps, persistent=1, replay=1, counters=None):
    g, p, L = make3(N, eta, cells, ell, nm, seed, persistent, replay)
    assert g.get_param(E.PARAM3_PERSISTENT) == persistent
    x, y, z = W.cubic_lattice(N, L)
    tot = oracle.Stats()
    for s in range(n_sweeps):
        cells_or = oracle.bin_cells3(p, s, x, y, z)
        st, recs = oracle.sweeps3(p, x, y, z, s, 1, stats=tot, records=True)
        g.sweep(1)
        assert np.array_equal(g.last_cells(), cells_or), "binning differs at sweep %d" % s
        gr = g.chain_records()
        orr = recs[0]
        assert np.array_equal(gr[:, :, 0], orr["start_id"]), "start spheres, sweep %d" % s
        ran = orr["start_id"] >= 0
        assert np.array_equal(gr[:, :, 1][ran], orr["end_id"][ran]), "end spheres, sweep %d" % s
        assert np.array_equal(gr[:, :, 2][ran], orr["events"][ran]), "events, sweep %d" % s
        assert np.array_equal(gr[:, :, 3][ran], orr["walls"][ran]), "walls, sweep %d" % s
        assert_positions_equal(g, x, y, z, L)
    c = g.counters()
    assert c.events == tot.events and c.lifts == tot.lifts
    assert c.frozen_hits == tot.frozen_hits and c.wall_hits == tot.wall_hits
    assert c.chains == tot.chains and c.sweeps == n_sweeps
    assert c.sum_b == pytest.approx(tot.sum_b, rel=1e-11, abs=1e-12)
    P_gpu, _ = g.pressure()
    P_or = oracle.pressure_from_sums3(tot.sum_b_w, tot.sum_disp_w, N, L, 1.0)
    assert P_gpu == pytest.approx(P_or, rel=1e-11)
    assert g.sweep_index() == n_sweeps
    if counters is not None:
        counters.append(c)
    g.close()
    return tot


@pytest.mark.parametrize("N,eta,cells,ell,nm,sweeps", [
    (64, 0.30, 2, 1.0, 4, 12),       # two cells per side: neighbours coincide
    (512, 0.45, 4, 0.8, 3, 8),
    (1000, 0.40, 4, 2.0, 5, 6),      # ragged member counts
    (4096, 0.50, 8, 1.5, 2, 4),
    (13824, 0.49, 10, 1.0, 1, 3),
    (8000, 0.30, 6, 3.0, 6, 3),
])
@pytest.mark.parametrize("persistent", [1, 0])
def test_sweeps_match_oracle(N, eta, cells, ell, nm, sweeps, persistent):
    st = run_pair3(N, eta, cells, ell, nm, 5, sweeps, persistent)
    assert st.events > 0 and st.frozen_hits > 0 and st.wall_hits > 0


def test_every_axis_and_a_long_run():
    # 9 sweeps cover the axes x, y, z three times each
    run_pair3(512, 0.52, 2, 1.2, 4, 8, 9)


def test_min_distance_and_overlap_check():
    N, eta, cells = 4096, 0.45, 8
    g, p, L = make3(N, eta, cells, 1.0, 3, 2)
    x, y, z = W.cubic_lattice(N, L)
    oracle.sweeps3(p, x, y, z, 0, 10)
    xyz = np.empty(3 * N)
    xyz[0::3], xyz[1::3], xyz[2::3] = x, y, z
    g.set_positions(xyz, t0=10)
    rc = min(2.0, L / cells)
    assert g.min_distance() == math.sqrt(oracle.min_dist2_3(L, x, y, z, rc))
    # move sphere 1 onto sphere 0 at distance 0.5: rejected
    bad = xyz.copy()
    bad[3:6] = bad[0:3] + np.array([0.5, 0.0, 0.0])
    with pytest.raises(E.EcmcError) as ei:
        g.set_positions(bad, t0=10)
    assert ei.value.code == E.ERR_OVERLAP
    # the handle recovers from the rejected input; sweeps keep spheres apart
    g.set_positions(xyz, t0=10)
    g.sweep(2)
    after = g.positions()
    x2, y2, z2 = after[0::3].copy(), after[1::3].copy(), after[2::3].copy()
    assert oracle.min_dist2_3(L, x2, y2, z2, rc) >= 1.0 - 1e-12
    assert g.min_distance() == math.sqrt(oracle.min_dist2_3(L, x2, y2, z2, rc))
    g.close()


def test_resume_from_positions_is_bitwise():
    N, eta, cells = 512, 0.45, 4
    g, p, L = make3(N, eta, cells, 1.0, 2, 4)
    g.sweep(6)
    ref = g.positions().copy()
    g.close()
    g, p, L = make3(N, eta, cells, 1.0, 2, 4)
    g.sweep(3)
    mid = g.positions().copy()
    g.close()
    g, p, L = make3(N, eta, cells, 1.0, 2, 4)
    g.set_positions(mid, t0=3)
    g.sweep(3)
    assert np.array_equal(g.positions(), ref)
    g.close()


def test_pressure_has_an_error_bar_and_resets():
    g, p, L = make3(1000, 0.3, 4, 2.0, 8, 6)
    g.sweep(100)
    P1, se = g.pressure()
    assert se > 0.0 and P1 > 0.0
    g.reset_stats()
    with pytest.raises(E.EcmcError):
        g.pressure()
    g.close()


def test_pressure_matches_carnahan_starling():
    # the CUDA path's own sampling at scale (not only its parity): eta = 0.3,
    # where the Carnahan-Starling equation is accurate to about 0.1 %
    N, eta = 4096, 0.30
    g, p, L = make3(N, eta, 6, 2.0, 20, 12)
    g.sweep(300)
    g.reset_stats()
    g.sweep(3000)
    P3, se = g.pressure()
    rho = N / L**3
    z, zse = P3 / rho, se / rho
    cs = (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3
    assert abs(z - cs) < 4.0 * zse + 0.003 * cs, (z, cs, zse)
    g.close()


@pytest.mark.parametrize("persistent", [1, 0])
def test_replayed_rattles_match_oracle(persistent):
    # cells of 2.1 sigma and chains of 2 sigma at eta = 0.45: a few chains
    # rattle between frozen spheres for hundreds of legs, and the replay of
    # their periodic legs must leave every sweep as the oracle's full search
    # does (binning, chain records, positions, counters, pressure)
    cs = []
    run_pair3(32768, 0.45, 16, 2.0, 1, 9, 10, persistent, replay=1, counters=cs)
    assert cs[0].replayed_legs > 0


def test_replay_on_and_off_are_bitwise_equal():
    a, p, L = make3(32768, 0.45, 16, 2.0, 1, 9, replay=1)
    b, p, L = make3(32768, 0.45, 16, 2.0, 1, 9, replay=0)
    assert a.get_param(E.PARAM3_REPLAY) == 1 and b.get_param(E.PARAM3_REPLAY) == 0
    a.sweep(20)
    b.sweep(20)
    assert np.array_equal(a.positions(), b.positions())
    ca, cb = a.counters(), b.counters()
    assert ca.events == cb.events and ca.lifts == cb.lifts and ca.sum_b == cb.sum_b
    assert ca.frozen_hits == cb.frozen_hits and ca.wall_hits == cb.wall_hits
    assert ca.replayed_legs > 0 and cb.replayed_legs == 0
    assert a.pressure()[0] == b.pressure()[0]
    a.close()
    b.close()


def test_persistent_and_per_phase_sweeps_are_bitwise_equal():
    a, p, L = make3(32768, 0.45, 16, 1.0, 3, 21, persistent=1)
    b, p, L = make3(32768, 0.45, 16, 1.0, 3, 21, persistent=0)
    a.sweep(12)
    b.sweep(12)
    assert np.array_equal(a.positions(), b.positions())
    ca, cb = a.counters(), b.counters()
    assert ca.events == cb.events and ca.sum_b == cb.sum_b
    a.close()
    b.close()


def test_dependency_wait_times_out_and_recovers():
    # the failure test: every wait looks for a value nobody writes and runs
    # out after 200 ms; the sweep reports a timeout, the handle recovers once
    # positions are set again (no device fault)
    g, p, L = make3(4096, 0.40, 8, 1.0, 2, 3)
    g.sweep(2)
    xyz = g.positions().copy()
    t = g.sweep_index()
    g.set_param(E.PARAM3_WAIT_LIMIT_MS, 200)
    g.set_param(E.PARAM3_WAIT_TEST, 1)
    g.sweep(1)
    with pytest.raises(E.EcmcError) as ei:
        g.synchronize()
    assert ei.value.code == E.ERR_TIMEOUT
    g.set_param(E.PARAM3_WAIT_TEST, 0)
    g.set_positions(xyz, t0=t)
    g.sweep(2)
    g.synchronize()
    ref, _, _ = make3(4096, 0.40, 8, 1.0, 2, 3)
    ref.sweep(4)
    assert np.array_equal(g.positions(), ref.positions())
    g.close()
    ref.close()


def test_handles_with_different_frame_sizes_coexist():
    # the kernels' shared-memory limit is process-wide: a handle with small
    # frames created after one with large frames must not break the latter
    big, pb, Lb = make3(4096, 0.45, 4, 1.0, 2, 31)      # cells of 4 sigma
    small, ps, Ls = make3(32768, 0.45, 16, 1.0, 2, 32)  # cells of 2 sigma
    small.sweep(2)
    big.sweep(2)
    small.sweep(1)
    big.synchronize()
    small.synchronize()
    x, y, z = W.cubic_lattice(4096, Lb)
    oracle.sweeps3(pb, x, y, z, 0, 2)
    assert_positions_equal(big, x, y, z, Lb)
    big.close()
    small.close()
