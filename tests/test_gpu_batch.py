"""Batches of independent replicas advanced in the same launches.

Each replica of a batch must follow exactly the trajectory the oracle gives
for its own parameters (N, eta, cells, ell, n_m, Philox key), whatever the
other replicas are; per-replica pressures are the oracle's member-weighted
collision estimator; FP32 screening and FP64 candidates give identical
batches (the pressure difference between the two forms is exactly zero).
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

REL = 1e-12

# heterogeneous replicas: sizes, densities, cell grids (incl. rectangular and
# two per side), displacements, chains per cell and keys all differ
REPLICAS = [
    dict(N=256, eta=0.70, cells_x=2, cells_y=2, ell=4.0, n_m=2, seed=1, replica=0),
    dict(N=1024, eta=0.72, cells_x=4, cells_y=8, ell=2.0, n_m=3, seed=1, replica=1),
    dict(N=4096, eta=0.65, cells_x=16, cells_y=16, ell=3.0, n_m=1, seed=9, replica=0),
    dict(N=576, eta=0.60, cells_x=6, cells_y=6, ell=5.0, n_m=2, seed=4, replica=7),
    dict(N=64, eta=0.05, cells_x=8, cells_y=8, ell=5.0, n_m=3, seed=11, replica=2),
]


def descs(reps):
    out = []
    for d in reps:
        e = dict(d)
        e["L"] = W.box_side(d["N"], d["eta"])
        out.append(e)
    return out


def oracle_run(d, n_sweeps):
    L = W.box_side(d["N"], d["eta"])
    x, y = W.square_lattice(d["N"], L)
    p = oracle.make_params(d["N"], L, 1.0, d["cells_x"], d["cells_y"], d["ell"], d["n_m"],
                           d["seed"], d["replica"])
    st, _ = oracle.sweeps(p, x, y, 0, n_sweeps)
    return x, y, st, L


@pytest.mark.parametrize("prec", [0, 1])
def test_every_replica_matches_its_oracle(prec):
    ds = descs(REPLICAS)
    g = P.Ecmc.batch(ds)
    g.set_param(E.PARAM_PRECISION, prec)
    g.sweep(4)
    xy = g.positions()
    off = 0
    for r, d in enumerate(REPLICAS):
        x, y, st, L = oracle_run(d, 4)
        gx = xy[2 * off: 2 * (off + d["N"]): 2]
        gy = xy[2 * off + 1: 2 * (off + d["N"]): 2]
        dx = np.abs(gx - x)
        dy = np.abs(gy - y)
        worst = max(np.minimum(dx, L - dx).max(), np.minimum(dy, L - dy).max()) / L
        assert worst <= REL, (r, worst)
        c = g.replica_counters(r)
        assert c.events == st.events and c.wall_hits == st.wall_hits and c.chains == st.chains
        rho = d["N"] / L**2
        Pg, _ = g.replica_pressure(r)
        assert Pg == pytest.approx(rho * (1 + st.sum_b_w / st.sum_disp_w), rel=1e-11)
        assert g.replica_desc(r)["n_m"] == d["n_m"]
        off += d["N"]
    tot = g.counters()
    assert tot.events == sum(g.replica_counters(r).events for r in range(len(REPLICAS)))
    g.close()


def test_batch_equals_separate_handles():
    ds = descs(REPLICAS[:3])
    g = P.Ecmc.batch(ds)
    g.sweep(3)
    xy = g.positions()
    off = 0
    for d in ds:
        s = P.Ecmc(d["N"], d["L"], 1.0, d["cells_x"], d["cells_y"], d["ell"], d["seed"])
        s.set_param(E.PARAM_N_CHAINS, d["n_m"])
        s.set_param(E.PARAM_REPLICA, d["replica"])
        s.sweep(3)
        assert np.array_equal(s.positions(), xy[2 * off: 2 * (off + d["N"])])
        off += d["N"]
        s.close()
    g.close()


def test_fp32_screening_pressure_error_is_zero():
    # the equation-of-state shape: several densities side by side
    reps = [dict(N=4096, eta=eta, cells_x=12, cells_y=12, ell=2.0, n_m=0, seed=6, replica=r)
            for r, eta in enumerate([0.69, 0.70, 0.71, 0.72, 0.73, 0.74])]
    ds = descs(reps)
    a = P.Ecmc.batch(ds)
    b = P.Ecmc.batch(ds)
    b.set_param(E.PARAM_PRECISION, 0)
    a.sweep(20)
    b.sweep(20)
    assert np.array_equal(a.positions(), b.positions())
    for r in range(len(reps)):
        assert a.replica_pressure(r)[0] == b.replica_pressure(r)[0]
    a.close()
    b.close()


def test_set_positions_for_the_whole_batch():
    ds = descs(REPLICAS[:2])
    g = P.Ecmc.batch(ds)
    g.sweep(2)
    mid = g.positions().copy()
    g.sweep(2)
    end = g.positions().copy()
    g.set_positions(mid, t0=2)
    g.sweep(2)
    assert np.array_equal(g.positions(), end)
    g.close()


def test_autotune_keeps_the_trajectory():
    N, eta = 4096, 0.72
    L = W.box_side(N, eta)
    a = P.Ecmc(N, L, 1.0, 16, 16, 2.0, 3)
    b = P.Ecmc(N, L, 1.0, 16, 16, 2.0, 3)
    a.sweep(2)
    b.sweep(2)
    best, shapes = a.autotune(trial_sweeps=2)
    assert len(shapes) >= 3 and best["ms_per_sweep"] == min(s["ms_per_sweep"] for s in shapes)
    # both the persistent sweep kernel and the per-phase kernels were timed
    assert {s["persistent"] for s in shapes} == {0, 1}
    assert a.get_param(E.PARAM_PERSISTENT) == best["persistent"]
    assert a.get_param(E.PARAM_LANES_PER_CELL) == best["lanes_per_cell"]
    assert a.sweep_index() == 2 and np.array_equal(a.positions(), b.positions())
    assert a.counters().sweeps == b.counters().sweeps
    a.sweep(3)
    b.sweep(3)
    assert np.array_equal(a.positions(), b.positions())
    a.close()
    b.close()


def test_every_replica_has_its_own_pair_histogram():
    # ecmc_replica_gr_measure(-1) adds each replica's configuration to its own
    # histogram: integer counts equal the oracle's pair counts of that replica
    ds = descs(REPLICAS[:4])
    g = P.Ecmc.batch(ds)
    g.set_param(E.PARAM_GR_DR, 0.02)
    g.set_param(E.PARAM_GR_RMAX, 3.0)
    nb = g.gr_nbins()
    g.sweep(3)
    g.gr_measure(-1)
    g.sweep(2)
    g.gr_measure(-1)
    g.gr_measure(1)
    for r, d in enumerate(REPLICAS[:4]):
        want = np.zeros(nb, np.int64)
        x, y, _, L = oracle_run(d, 3)
        oracle.gr_counts(L, x, y, 1.0, 0.02, nb, counts=want)
        p = oracle.make_params(d["N"], L, 1.0, d["cells_x"], d["cells_y"], d["ell"], d["n_m"],
                               d["seed"], d["replica"])
        oracle.sweeps(p, x, y, 3, 2)
        oracle.gr_counts(L, x, y, 1.0, 0.02, nb, counts=want)
        if r == 1:
            oracle.gr_counts(L, x, y, 1.0, 0.02, nb, counts=want)
        got, n_meas = g.gr_counts(r)
        assert n_meas == (3 if r == 1 else 2)
        assert np.array_equal(got, want), r
    g.close()
