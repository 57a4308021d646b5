"""Long runs of the CUDA sweep against the oracle and against closed forms.

The chain-estimator pressure and g(r) of independent runs (different Philox
seeds) must agree within 3 combined standard errors; the low-density pressure
must follow the virial series of hard disks.
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

from test_oracle_pressure import virial  # noqa: E402


def gpu_batches(N, eta, cells, ell, nm, seed, n_batches, per_batch, warm, gr_every=0, dr=0.02,
                nbins=10, dir_mode=0):
    L = W.box_side(N, eta)
    g = P.Ecmc(N, L, 1.0, cells, cells, ell, seed)
    g.set_param(E.PARAM_N_CHAINS, nm)
    g.set_param(E.PARAM_DIR_MODE, dir_mode)
    g.set_param(E.PARAM_GR_DR, dr)
    g.set_param(E.PARAM_GR_RMAX, 1.0 + dr * nbins)
    g.sweep(warm)
    vals, grs = [], []
    for _ in range(n_batches):
        g.reset_stats()
        if gr_every:
            for _ in range(per_batch // gr_every):
                g.sweep(gr_every)
                g.gr_measure()
            _, gb = g.gr()
            grs.append(gb)
        else:
            g.sweep(per_batch)
        p, _ = g.pressure()
        vals.append(p)
    g.close()
    vals = np.array(vals)
    return vals.mean(), vals.std(ddof=1) / math.sqrt(n_batches), np.array(grs)


def oracle_batches(N, eta, cells, ell, nm, seed, n_batches, per_batch, warm, gr_every=0,
                   dr=0.02, nbins=10):
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, cells, cells, ell, nm, seed)
    oracle.sweeps(p, x, y, 0, warm)
    t = warm
    vals, grs = [], []
    rho = N / L**2
    for _ in range(n_batches):
        st = oracle.Stats()
        counts = np.zeros(nbins, np.int64)
        nmeas = 0
        if gr_every:
            for _ in range(per_batch // gr_every):
                oracle.sweeps(p, x, y, t, gr_every, stats=st)
                t += gr_every
                oracle.gr_counts(L, x, y, 1.0, dr, nbins, counts=counts)
                nmeas += 1
            grs.append(oracle.gr_normalise(counts, nmeas, N, L, 1.0, dr)[1])
        else:
            oracle.sweeps(p, x, y, t, per_batch, stats=st)
            t += per_batch
        vals.append(rho * (1.0 + st.sum_b_w / st.sum_disp_w))
    vals = np.array(vals)
    return vals.mean(), vals.std(ddof=1) / math.sqrt(n_batches), np.array(grs)


def test_pressure_and_gr_agree_with_oracle_across_seeds():
    # 1024 disks at eta = 0.65 (liquid), 4x4 cells, ell = 4, n_m = 2
    args = (1024, 0.65, 4, 4.0, 2)
    Pg, sg, gg = gpu_batches(*args, seed=101, n_batches=20, per_batch=300, warm=300, gr_every=10)
    Po, so, go = oracle_batches(*args, seed=202, n_batches=20, per_batch=300, warm=300,
                                gr_every=10)
    assert abs(Pg - Po) < 3.0 * math.hypot(sg, so), (Pg, sg, Po, so)
    mg, mo = gg.mean(0), go.mean(0)
    eg = gg.std(0, ddof=1) / math.sqrt(len(gg))
    eo = go.std(0, ddof=1) / math.sqrt(len(go))
    z = (mg - mo) / np.hypot(eg, eo)
    assert np.mean(z**2) < 3.0 and np.max(np.abs(z)) < 4.0, z


@pytest.mark.parametrize("eta,cells", [(0.05, 4), (0.10, 8)])
def test_low_density_pressure_matches_virial_series(eta, cells):
    N = 256
    L = W.box_side(N, eta)
    rho = N / L**2
    Pv = rho * virial(eta)
    Pg, sg, _ = gpu_batches(N, eta, cells, 20.0, 4, 77, n_batches=20, per_batch=200, warm=200)
    assert abs(Pg - Pv) < 4.0 * sg, (Pg, sg, Pv)
    assert abs(Pg - rho * (1 + 2 * eta)) > 10.0 * sg


def test_pressure_error_bar_is_batch_means():
    N, eta = 1024, 0.70
    L = W.box_side(N, eta)
    g = P.Ecmc(N, L, 1.0, 4, 4, 4.0, 3)
    g.sweep(100)
    g.reset_stats()
    g.sweep(400)
    p, se = g.pressure()
    rho = N / L**2
    assert se > 0 and se < 0.05 * p and p > rho
    g.close()


def test_isotropic_and_axis_chains_sample_the_same_pressure():
    # both direction rules are reversible and sample the uniform measure
    # (Sec. 3.2-3.4): independent runs must agree within 3 combined errors
    args = (1024, 0.68, 4, 3.0, 2)
    Pa, sa, _ = gpu_batches(*args, seed=31, n_batches=20, per_batch=300, warm=300)
    Pi, si, _ = gpu_batches(*args, seed=32, n_batches=20, per_batch=300, warm=300, dir_mode=2)
    assert abs(Pa - Pi) < 3.0 * math.hypot(sa, si), (Pa, sa, Pi, si)

