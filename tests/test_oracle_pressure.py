"""Pins (c) of the oracle's pressure estimators.

The collision estimator beta P / rho = 1 + sum_b / sum_disp is the collision
form of eq. (pressure) (Sec. 2; the extension to the cell-decomposed sweep is
left open at the end of Sec. 3.4).  Because every cell receives the same
displacement n_m ell whatever its number of members n_c, the per-cell sums
are weighted by n_c; the unweighted sums are biased low.  Pinned against the
low-density virial series of hard disks and against the textbook sequential
event chain without cells (Sec. 3.2)."""
import math
import os

import numpy as np
import pytest

import ecmc_workloads as W
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def virial_coeffs():
    vals = {}
    with open(os.path.join(HERE, "golden", "hard_disk_virial.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_virial_golden_matches_closed_forms():
    v = virial_coeffs()
    assert v["B3_over_B2sq"] == pytest.approx(4.0 / 3.0 - math.sqrt(3.0) / math.pi, abs=1e-9)
    assert v["B4_over_B2cu"] == pytest.approx(
        2.0 - 9.0 * math.sqrt(3.0) / (2.0 * math.pi) + 10.0 / math.pi**2, abs=1e-9)


def virial(eta):
    v = virial_coeffs()
    b2rho = 2.0 * eta
    return 1.0 + b2rho + v["B3_over_B2sq"] * b2rho**2 + v["B4_over_B2cu"] * b2rho**3


def pec_batches(N, eta, cells, ell, nm, n_batches, per_batch, warm, seed=11):
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, cells, cells, ell, nm, seed)
    oracle.sweeps(p, x, y, 0, warm)
    w, u = [], []
    for b in range(n_batches):
        st, _ = oracle.sweeps(p, x, y, warm + b * per_batch, per_batch)
        w.append(st.sum_b_w / st.sum_disp_w)
        u.append(st.sum_b / st.sum_disp)
    w, u = np.array(w), np.array(u)
    se = lambda a: a.std(ddof=1) / math.sqrt(len(a))
    return 1 + w.mean(), se(w), 1 + u.mean(), se(u)


@pytest.mark.parametrize("eta,cells,ell", [(0.05, 4, 20.0), (0.10, 8, 20.0)])
def test_low_density_matches_virial_series(eta, cells, ell):
    P, se, Pu, seu = pec_batches(256, eta, cells, ell, 4, 20, 200, 200)
    # the B4 truncation error (B5 term ~ 5 eta^4) is far below the error bar
    assert abs(P - virial(eta)) < 4.0 * se
    # the third virial coefficient is resolved: B2 alone is rejected
    assert abs(P - (1.0 + 2.0 * eta)) > 10.0 * se


def test_unweighted_cell_sums_are_biased():
    # equal displacement per cell over-weights sparsely filled cells
    P, se, Pu, seu = pec_batches(256, 0.10, 8, 20.0, 4, 20, 200, 200)
    assert (virial(0.10) - Pu) > 10.0 * seu


def test_sequential_chain_matches_virial_series():
    eta, N = 0.05, 256
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    oracle.seq_sweeps(N, L, 1.0, 20.0, 64, 11, 0, x, y, 0, 100)
    vals = []
    for b in range(20):
        st = oracle.seq_sweeps(N, L, 1.0, 20.0, 64, 11, 0, x, y, 100 + b * 60, 60)
        vals.append(st.sum_b / st.sum_disp)
    vals = np.array(vals)
    P, se = 1 + vals.mean(), vals.std(ddof=1) / math.sqrt(len(vals))
    assert abs(P - virial(eta)) < 4.0 * se


def test_dense_cell_sweep_matches_sequential_chain():
    eta, N = 0.60, 256
    P, se, _, _ = pec_batches(N, eta, 4, 4.0, 1, 20, 400, 500)
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    oracle.seq_sweeps(N, L, 1.0, 4.0, 16, 11, 0, x, y, 0, 500)
    vals = []
    for b in range(20):
        st = oracle.seq_sweeps(N, L, 1.0, 4.0, 16, 11, 0, x, y, 500 + b * 200, 200)
        vals.append(st.sum_b / st.sum_disp)
    vals = np.array(vals)
    Ps, ses = 1 + vals.mean(), vals.std(ddof=1) / math.sqrt(len(vals))
    assert abs(P - Ps) < 4.0 * math.hypot(se, ses)
