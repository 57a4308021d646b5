"""Parity of the CUDA sweep with the oracle, through the C ABI.

The CUDA path evaluates every contact with the same FP64 expressions as the
oracle (FP64 without contraction on both sides, IEEE division and square
root), so trajectories agree to the last bit; the tests allow 1e-12 relative
on positions (the bar for the first ten sweeps of the N = 256 system) and
compare integer results (cells, counters, chain records, pair counts)
exactly.  Cases span several frame sizes, ragged cell counts, lanes per cell
1..32, both candidate-screening modes, empty cells and the degenerate ones.
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
LAST = {}  # counters of the most recent run_pair, for tests that inspect them


def make(N, eta, cells_x, cells_y, ell, nm, seed, tpc=0, prec=1, dir_mode=0, records=False,
         replica=0, fmode=-1, persistent=1, list_mode=0, boundary=0):
    L = W.box_side(N, eta)
    g = P.Ecmc(N, L, 1.0, cells_x, cells_y, ell, seed)
    g.set_param(E.PARAM_N_CHAINS, nm)
    g.set_param(E.PARAM_PRECISION, prec)
    g.set_param(E.PARAM_DIR_MODE, dir_mode)
    g.set_param(E.PARAM_REPLICA, replica)
    if tpc:
        g.set_param(E.PARAM_LANES_PER_CELL, tpc)
    if fmode >= 0:
        g.set_param(E.PARAM_FRAME_MODE, fmode)
    g.set_param(E.PARAM_PERSISTENT, persistent)
    g.set_param(E.PARAM_LIST_MODE, list_mode)
    if boundary:
        g.set_param(E.PARAM_BOUNDARY, boundary)
    if records:
        g.set_param(E.PARAM_RECORD_CHAINS, 1)
    p = oracle.make_params(N, L, 1.0, cells_x, cells_y, ell, nm, seed, replica,
                           dir_mode=dir_mode, list_mode=list_mode, boundary=boundary)
    return g, p, L


def assert_positions_equal(g, x, y, L):
    xy = g.positions()
    gx, gy = xy[0::2], xy[1::2]
    # equal up to the periodic wrap
    dx = np.abs(gx - x)
    dx = np.minimum(dx, L - dx)
    dy = np.abs(gy - y)
    dy = np.minimum(dy, L - dy)
    worst = max(dx.max(), dy.max()) / L
    assert worst <= REL, "max relative position difference %g" % worst
    return worst


def run_pair(N, eta, cells_x, cells_y, ell, nm, seed, n_sweeps, records=True, **kw):
    g, p, L = make(N, eta, cells_x, cells_y, ell, nm, seed, records=records, **kw)
    x, y = W.square_lattice(N, L)
    st_total = oracle.Stats()
    for s in range(n_sweeps):
        cells_or = oracle.bin_cells(p, s, x, y)
        st, recs = oracle.sweeps(p, x, y, s, 1, stats=st_total, records=records)
        g.sweep(1)
        assert np.array_equal(g.last_cells(), cells_or), "binning differs at sweep %d" % s
        if records:
            gr = g.chain_records()
            orr = recs[0]
            assert np.array_equal(gr["start_id"], orr["start_id"]), "start disks, sweep %d" % s
            assert np.array_equal(gr["end_id"], orr["end_id"]), "end disks, sweep %d" % s
            ran = orr["start_id"] >= 0  # cells without members start no chain
            assert np.array_equal(gr["events"][ran], orr["events"][ran]), "events, sweep %d" % s
            assert np.array_equal(gr["walls"][ran], orr["walls"][ran]), "walls, sweep %d" % s
        assert_positions_equal(g, x, y, L)
    c = g.counters()
    LAST["counters"] = c.as_dict()
    assert c.events == st_total.events and c.lifts == st_total.lifts
    assert c.frozen_hits == st_total.frozen_hits and c.wall_hits == st_total.wall_hits
    assert c.chains == st_total.chains and c.sweeps == n_sweeps
    assert c.rejected_chains == st_total.rejected
    assert c.sum_b == pytest.approx(st_total.sum_b, rel=1e-11, abs=1e-12)
    # the oracle adds ell chain by chain, the library multiplies a count by ell
    assert c.sum_disp == pytest.approx(st_total.sum_disp, rel=1e-11)
    if st_total.sum_disp_w > 0:
        P_gpu, _ = g.pressure()
        rho = N / L**2
        P_or = rho * (1.0 + st_total.sum_b_w / st_total.sum_disp_w)
        assert P_gpu == pytest.approx(P_or, rel=1e-11)
    g.close()
    return st_total


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("tpc", [1, 2, 4, 8, 16, 32])
def test_small_system_ten_sweeps(tpc, prec):
    # 256 disks at eta = 0.70, 2x2 cells, ell = 4 sigma, n_m = 2: the
    # two-cells-per-side case where one neighbour supplies both halos
    st = run_pair(256, 0.70, 2, 2, 4.0, 2, 1, 10, tpc=tpc, prec=prec)
    assert st.events > 1000 and st.frozen_hits > 0


def test_wall_reflections_and_many_sweeps():
    # smaller cells and longer chains: wall reflections on every sweep
    st = run_pair(1024, 0.70, 8, 8, 6.0, 2, 13, 12)
    assert st.wall_hits > 0 and st.frozen_hits > 0


@pytest.mark.parametrize("N,eta,cx,cy,ell,nm,tpc", [
    (1024, 0.72, 4, 4, 8.0, 2, 0),
    (1024, 0.72, 8, 8, 2.0, 1, 4),
    (4096, 0.72, 16, 16, 2.0, 1, 1),
    (4096, 0.72, 4, 8, 4.0, 3, 2),     # ragged: rectangular cells
    (2304, 0.65, 6, 12, 3.0, 5, 8),    # 48^2 disks, cells not a power of two
    (65536, 0.708, 32, 32, 8.0, 1, 0),
])
def test_medium_systems(N, eta, cx, cy, ell, nm, tpc):
    run_pair(N, eta, cx, cy, ell, nm, 7, 3, tpc=tpc)


def test_positive_only_direction_rule():
    run_pair(1024, 0.70, 4, 4, 4.0, 2, 3, 4, dir_mode=1)


@pytest.mark.parametrize("N,eta,cx,ell,nm,tpc", [
    (256, 0.70, 2, 4.0, 2, 8),     # two cells per side
    (1024, 0.70, 8, 6.0, 2, 4),    # chains longer than a cell: many wall reflections
    (4096, 0.72, 16, 2.0, 1, 32),
    (1024, 0.30, 4, 3.0, 3, 0),    # dilute, automatic lanes per cell
])
@pytest.mark.parametrize("prec,persistent", [(1, 1), (0, 0), (1, 0)])
def test_isotropic_directions(N, eta, cx, ell, nm, tpc, prec, persistent):
    # uniform directions per chain, specular reflection at frozen disks (Fig. 1);
    # FP32-screened or all-FP64 candidates, persistent or per-phase launches
    st = run_pair(N, eta, cx, cx, ell, nm, 7, 5, tpc=tpc, dir_mode=2, prec=prec,
                  persistent=persistent)
    assert st.frozen_hits > 0 and st.wall_hits > 0


@pytest.mark.parametrize("N,eta,cx,ell,nm,dir_mode,persistent", [
    (1024, 0.70, 8, 4.0, 3, 0, 1),   # n_m < members: a prefix of the shuffled list
    (64, 0.05, 8, 5.0, 3, 0, 1),     # about one member per cell: the list cycles
    (1024, 0.70, 8, 4.0, 20, 0, 0),  # n_m > members, per-phase kernels
    (1024, 0.70, 8, 4.0, 3, 2, 0),   # isotropic directions
])
def test_shuffled_start_lists(N, eta, cx, ell, nm, dir_mode, persistent):
    # the negative control of Sec. 3.4: start lists without replacement
    run_pair(N, eta, cx, cx, ell, nm, 9, 4, dir_mode=dir_mode, persistent=persistent,
             list_mode=1)


def test_replica_key_changes_the_stream():
    st = run_pair(1024, 0.70, 4, 4, 4.0, 2, 3, 2, replica=5)
    assert st.chains == 2 * 16 * 2


def test_sparse_system_with_empty_cells():
    # 64 disks, 8x8 cells at eta = 0.05: many cells hold no disk
    run_pair(64, 0.05, 8, 8, 5.0, 3, 11, 6)


def test_single_disk():
    run_pair(1, 0.01, 2, 2, 3.0, 2, 4, 5)


def test_zero_displacement():
    st = run_pair(256, 0.70, 2, 2, 0.0, 1, 1, 3)
    assert st.events == 0


def test_large_system_full_size_two_sweeps():
    # the benchmark workload: 1024^2 disks at eta = 0.72 with the launch
    # configuration the benchmark times (automatic lanes per cell, FP32
    # screening); every position compared after each sweep
    N = 1048576
    run_pair(N, 0.72, 128, 128, 8.0, 1, 3, 2, records=False)


def test_replayed_reflections_at_the_paper_parameters():
    # 1024^2 disks at eta = 0.72 with the paper's cells, ell and n_m after a
    # melt: the regime where disks rattle between frozen neighbours for
    # hundreds of legs; every position compared after each sweep
    N, eta = 1048576, 0.72
    L = W.box_side(N, eta)
    par = E.suggest_parameters(N, L)
    g, p, _ = make(N, eta, par["cells_x"], par["cells_y"], par["ell"], par["n_m"], 8)
    x, y = W.square_lattice(N, L)
    oracle.sweeps(p, x, y, 0, 6)
    g.sweep(6)
    assert_positions_equal(g, x, y, L)
    st, _ = oracle.sweeps(p, x, y, 6, 2)
    g.reset_stats()
    g.sweep(2)
    assert_positions_equal(g, x, y, L)
    c = g.counters()
    assert c.events == st.events and c.frozen_hits == st.frozen_hits
    assert c.wall_hits == st.wall_hits and c.lifts == st.lifts
    assert c.replayed_legs > 0, c.replayed_legs
    g.close()


def test_gr_counts_and_min_distance_match():
    N, eta = 4096, 0.70
    g, p, L = make(N, eta, 8, 8, 4.0, 1, 21)
    x, y = W.square_lattice(N, L)
    oracle.sweeps(p, x, y, 0, 6)
    g.sweep(6)
    assert_positions_equal(g, x, y, L)
    g.gr_measure()
    counts, nm = g.gr_counts()
    ref = oracle.gr_counts(L, x, y, 1.0, 0.01, 400)
    assert nm == 1 and np.array_equal(counts, ref)
    assert g.min_distance() == pytest.approx(math.sqrt(oracle.min_dist2(L, x, y)), rel=1e-15)
    r, gr = g.gr()
    R, gor = oracle.gr_normalise(ref, 1, N, L, 1.0, 0.01)
    assert np.allclose(r, R, rtol=1e-14) and np.allclose(gr, gor, rtol=1e-13)
    g.close()


def test_resume_from_positions_is_bitwise():
    N, eta = 1024, 0.72
    g, p, L = make(N, eta, 4, 4, 4.0, 2, 9)
    g.sweep(3)
    mid = g.positions().copy()
    g.sweep(4)
    end = g.positions().copy()
    g.set_positions(mid, t0=3)
    assert g.sweep_index() == 3
    g.sweep(4)
    assert np.array_equal(g.positions(), end)
    g.close()


def test_device_pointer_io_and_stream():
    N, eta = 1024, 0.70
    g, p, L = make(N, eta, 4, 4, 4.0, 1, 2)
    s = torch.cuda.Stream()
    g.set_stream(s)
    x, y = W.square_lattice(N, L)
    xy = torch.tensor(np.stack([x, y], 1).ravel(), dtype=torch.float64, device="cuda")
    g.set_positions(xy, t0=0)
    g.sweep(2)
    out = torch.empty(2 * N, dtype=torch.float64, device="cuda")
    g.positions(out)
    torch.cuda.synchronize()
    oracle.sweeps(p, x, y, 0, 2)
    o = out.cpu().numpy()
    assert np.max(np.abs(o[0::2] - x)) < REL * L and np.max(np.abs(o[1::2] - y)) < REL * L
    g.set_stream(None)
    g.close()


def test_overlapping_input_is_rejected():
    N, eta = 256, 0.70
    g, p, L = make(N, eta, 2, 2, 4.0, 1, 2)
    x, y = W.square_lattice(N, L)
    x[1] = x[0] + 0.5
    y[1] = y[0]
    with pytest.raises(E.EcmcError) as ei:
        g.set_positions(np.stack([x, y], 1).ravel())
    assert ei.value.code == E.ERR_OVERLAP
    with pytest.raises(E.EcmcError) as ei:
        g.sweep(1)
    assert ei.value.code == E.ERR_STATE
    g.close()


def test_graph_replay_equals_direct_launches():
    N, eta = 4096, 0.72
    a, _, L = make(N, eta, 16, 16, 2.0, 1, 5)
    b, _, _ = make(N, eta, 16, 16, 2.0, 1, 5)
    b.set_param(E.PARAM_USE_GRAPH, 0)
    a.sweep(5)
    b.sweep(5)
    assert np.array_equal(a.positions(), b.positions())
    a.close()
    b.close()


@pytest.mark.parametrize("N,eta,cells,ell,nm", [
    (4096, 0.72, 2, 4.0, 8),      # 33-sigma cells: one cell per warp, frame in shared memory
    (16384, 0.72, 2, 4.0, 20),    # 67-sigma cells: frame used in global memory, staged builder
])
def test_large_cells(N, eta, cells, ell, nm):
    run_pair(N, eta, cells, cells, ell, nm, 5, 2)


@pytest.mark.parametrize("replay", [0, 1])
def test_replay_switch_gives_identical_trajectories(replay):
    # 1024 disks, 8x8 cells, ell = 6 sigma: chains cross whole cells and
    # rattle between walls and frozen disks; both settings match the oracle
    g, p, L = make(1024, 0.70, 8, 8, 6.0, 2, 13)
    g.set_param(E.PARAM_REPLAY, replay)
    x, y = W.square_lattice(1024, L)
    st, _ = oracle.sweeps(p, x, y, 0, 12)
    g.sweep(12)
    assert_positions_equal(g, x, y, L)
    c = g.counters()
    assert c.events == st.events and c.wall_hits == st.wall_hits
    assert (c.replayed_legs > 0) == bool(replay)
    g.close()


@pytest.mark.parametrize("fmode", [0, 1, 2])
@pytest.mark.parametrize("tpc", [1, 4, 32])
def test_frame_placements(fmode, tpc):
    # per-phase launches with frames in shared memory, FP64 part in global
    # memory, all in global memory
    run_pair(4096, 0.72, 16, 16, 3.0, 2, 17, 3, tpc=tpc, fmode=fmode, persistent=0)


@pytest.mark.parametrize("N,eta,cx,cy,ell,nm,tpc", [
    (256, 0.70, 2, 2, 4.0, 2, 8),      # two cells per side: neighbours coincide
    (1024, 0.70, 8, 8, 6.0, 2, 4),     # chains across whole cells, rattles
    (4096, 0.72, 4, 8, 4.0, 3, 8),     # rectangular cells, 128 disks each
    (4096, 0.72, 16, 16, 2.0, 1, 32),  # one cell per warp
])
@pytest.mark.parametrize("fmode", [0, 1])
def test_persistent_sweep_matches_oracle(N, eta, cx, cy, ell, nm, tpc, fmode):
    # one launch per sweep: work list over (phase, group) with waits on the
    # neighbours of earlier phases; frames wholly in shared memory (0) or FP64
    # coordinates in a per-warp global scratch area (1)
    g, _, _ = make(N, eta, cx, cy, ell, nm, 7, tpc=tpc, fmode=fmode)
    assert g.get_param(E.PARAM_PERSISTENT) == 1
    assert g.get_param(E.PARAM_FRAME_MODE) == fmode
    assert g.get_param(E.PARAM_KERNELS_PER_SWEEP) == 5
    g.close()
    run_pair(N, eta, cx, cy, ell, nm, 7, 4, tpc=tpc, fmode=fmode)


def test_persistent_and_phase_launches_are_bitwise_equal():
    N, eta = 65536, 0.708
    a, _, L = make(N, eta, 32, 32, 8.0, 1, 2)
    b, _, _ = make(N, eta, 32, 32, 8.0, 1, 2, persistent=0)
    assert a.get_param(E.PARAM_PERSISTENT) == 1 and b.get_param(E.PARAM_PERSISTENT) == 0
    a.sweep(6)
    b.sweep(6)
    assert np.array_equal(a.positions(), b.positions())
    assert a.counters().as_dict() == b.counters().as_dict()
    a.close()
    b.close()


def test_dependency_wait_timeout_is_reported_and_recoverable():
    # the waits of the persistent kernel look for a value nobody writes: every
    # wait runs into a 20 ms limit, the sweep is abandoned with a timeout
    # status the host reads, and the handle works again once positions are set
    N, eta = 4096, 0.72
    g, p, L = make(N, eta, 16, 16, 2.0, 1, 5)
    x, y = W.square_lattice(N, L)
    g.set_param(E.PARAM_WAIT_LIMIT_MS, 20.0)
    g.set_param(E.PARAM_WAIT_TEST, 1)
    with pytest.raises(E.EcmcError) as ei:
        g.sweep(1)
        g.positions()
    assert ei.value.code == E.ERR_TIMEOUT
    with pytest.raises(E.EcmcError) as ei:
        g.sweep(1)
    assert ei.value.code == E.ERR_STATE
    g.set_param(E.PARAM_WAIT_TEST, 0)
    g.set_positions(np.stack([x, y], 1).ravel(), t0=0)
    g.sweep(3)
    oracle.sweeps(p, x, y, 0, 3)
    assert_positions_equal(g, x, y, L)
    g.close()
