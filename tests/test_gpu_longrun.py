"""Long runs of the CUDA sweep against long runs of the oracle, on the small
(N = 256) and medium (N = 65,536) workloads at their full length.

Two checks per workload, from one GPU batch and one set of oracle runs:

1. Same keys.  The GPU batch also runs the oracle's own Philox keys; over the
   whole run those replicas must end at the oracle's positions (1e-12
   relative), with the oracle's g(r) counts exactly and its pressure to
   1e-10 relative.

2. Independent keys.  K_gpu further GPU runs (replicas 0..) against the
   oracle's K_oracle runs (replicas 1000..).  Both start from the same square
   lattice and apply the same transition rule, so at every sweep their
   configurations have the same distribution, whether or not the runs have
   equilibrated: the run averages of any observable have the same mean and
   run-to-run variance.  The difference of the two means is divided by its
   standard error from the pooled run-to-run variance (K_gpu + K_oracle - 2
   degrees of freedom).  Observables: the collision-form pressure (eq.
   pressure with the member-weighted chain sums) over the measured sweeps, and
   g(r) in 0.01 sigma bins from sigma to 5 sigma (Sec. 2), measured every 10
   sweeps.  Criteria: pressure within 3 combined standard errors; over the
   g(r) bins, mean z^2 below 3 and max |z| below 4.

The oracle runs go to a process pool started with spawn (before the GPU
side is launched), one run per host core, timed beside the GPU runs.
"""
import math
import multiprocessing as mp
import os
import time

import numpy as np
import pytest

import ecmc_workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1409_6948_gb300 as P  # noqa: E402
from paper_1409_6948_gb300 import ecmc as E  # noqa: E402

import longrun_oracle  # noqa: E402

DR, NBINS, GR_EVERY = 0.01, 400, 10
ORACLE_REPLICA0 = 1000


def gpu_runs(N, eta, cells, ell, n_m, seed, replicas, melt, sweeps):
    L = W.box_side(N, eta)
    g = P.Ecmc.batch([dict(N=N, L=L, cells_x=cells, ell=ell, n_m=n_m, seed=seed, replica=r)
                      for r in replicas])
    g.set_param(E.PARAM_GR_DR, DR)
    g.set_param(E.PARAM_GR_RMAX, 1.0 + DR * NBINS)
    assert g.gr_nbins() == NBINS
    t0 = time.time()
    g.sweep(melt)
    g.reset_stats()
    for _ in range(sweeps // GR_EVERY):
        g.sweep(GR_EVERY)
        g.gr_measure(-1)
    K = len(replicas)
    Pr = np.array([g.replica_pressure(r)[0] for r in range(K)])
    counts = np.array([g.gr_counts(r)[0] for r in range(K)])
    n_meas = g.gr_counts(0)[1]
    xy = g.positions().reshape(K, N, 2)
    ev = g.counters().events
    seconds = time.time() - t0
    g.close()
    return Pr, counts, n_meas, xy, ev, seconds


def pooled_z(a, b):
    """(mean a - mean b) / SE of the difference, SE from the pooled
    run-to-run variance."""
    ka, kb = a.shape[0], b.shape[0]
    va, vb = a.var(0, ddof=1), b.var(0, ddof=1)
    sp2 = ((ka - 1) * va + (kb - 1) * vb) / (ka + kb - 2)
    se = np.sqrt(sp2 * (1.0 / ka + 1.0 / kb))
    return (a.mean(0) - b.mean(0)) / se, se


def compare(name, N, eta, cells, ell, n_m, seed, K_gpu, K_orc, melt, sweeps):
    L = W.box_side(N, eta)
    ctx = mp.get_context("spawn")
    workers = max(1, min(K_orc, (os.cpu_count() or 2) - 1))
    args = [(N, eta, cells, ell, n_m, seed, ORACLE_REPLICA0 + r, melt, sweeps, GR_EVERY, DR,
             NBINS) for r in range(K_orc)]
    replicas = list(range(K_gpu)) + [ORACLE_REPLICA0 + r for r in range(K_orc)]
    t0 = time.time()
    with ctx.Pool(workers) as pool:
        pending = pool.starmap_async(longrun_oracle.run, args)
        Pg, cg, nmg, xy, ev_g, t_gpu = gpu_runs(N, eta, cells, ell, n_m, seed, replicas, melt,
                                                sweeps)
        orc = pending.get()
    t_orc = time.time() - t0
    ev_o = sum(o["events"] for o in orc)

    # 1. the oracle's keys on the GPU: the oracle's runs, to the last bit
    worst = 0.0
    for r, o in enumerate(orc):
        q = K_gpu + r
        for a, ref in ((0, o["x"]), (1, o["y"])):
            d = np.abs(xy[q, :, a] - ref)
            worst = max(worst, float((np.minimum(d, L - d)).max()) / L)
        assert np.array_equal(cg[q], o["counts"]) and nmg == o["n_meas"], r
        assert abs(Pg[q] - o["P"]) <= 1e-10 * o["P"], (r, Pg[q], o["P"])
    assert worst <= 1e-12, worst

    # 2. independent keys: statistical agreement
    Pi, Po = Pg[:K_gpu], np.array([o["P"] for o in orc])
    ci = cg[:K_gpu] / float(nmg)
    co = np.array([o["counts"] / float(o["n_meas"]) for o in orc])
    zp, sep = pooled_z(Pi, Po)
    ok = co.sum(0) > 0
    zg, _ = pooled_z(ci[:, ok], co[:, ok])
    chi2 = float(np.mean(zg**2))
    imax = int(np.argmax(np.abs(zg)))
    zmax = float(abs(zg[imax]))
    print("\n[%s] same keys: %d runs equal to the oracle (max rel %.1e) | independent: pressure "
          "gpu %.5f (K=%d) oracle %.5f (K=%d) diff %.5f se %.5f z %.2f | g(r) %d bins chi2/bin "
          "%.3f max|z| %.2f at r = %.3f | gpu %.1f s %.3g events/s | oracle %.1f s on %d "
          "processes %.3g events/s"
          % (name, K_orc, worst, Pi.mean(), K_gpu, Po.mean(), K_orc, Pi.mean() - Po.mean(),
             float(sep), float(zp), int(ok.sum()), chi2, zmax, 1.0 + DR * (imax + 0.5), t_gpu,
             ev_g / t_gpu, t_orc, workers, ev_o / t_orc))
    assert abs(zp) < 3.0, (Pi.mean(), Po.mean(), sep)
    assert chi2 < 3.0 and zmax < 4.0, (chi2, zmax)


def test_small_workload_1000_sweeps():
    # N = 256 at eta = 0.70, 2x2 cells, ell = 4 sigma, n_m = 2, Philox seed 1,
    # 1000 sweeps from the lattice
    compare("N=256", 256, 0.70, 2, 4.0, 2, 1, K_gpu=64, K_orc=64, melt=0, sweeps=1000)


def test_medium_workload_10000_sweeps():
    # N = 65,536 at eta = 0.708, 32x32 cells, ell = 8 sigma, n_m = 1 (eq. nm),
    # Philox seed 2, 100 melting sweeps then 10,000 measured sweeps
    compare("N=65536", 65536, 0.708, 32, 8.0, 1, 2, K_gpu=90, K_orc=15, melt=100,
            sweeps=10000)
