"""Pins of the oracle's rejecting boundary rule (ORC_BOUNDARY_REJECT), the
variant the paper compares its reflecting rule against (Sec. 3.4, Fig. 3):
a chain that reaches a cell wall or a frozen disk is rejected as a whole.

  - closed forms on hand-built frames: a chain whose budget ends inside the
    cell is accepted and equals the reflecting rule's result; one that lifts
    and then reaches a wall or a frozen disk leaves every coordinate exactly
    as it was, counts one rejection and adds nothing to sum_b or sum_disp;
    a budget ending exactly on the wall is accepted (chain end before wall);
  - one disk per cell, with the chain's sign recomputed from Philox: the
    result is x +- ell when the budget fits between the disk and the wall
    ahead, else x, bit for bit;
  - a budget longer than the cell's diagonal can never be spent inside the
    cell, so every chain is rejected and the configuration is unchanged;
  - three disks, 2x2 cells: chains started with replacement still sample
    the uniform measure (the exact pair-distance distribution of
    tests/threedisk_exact.py), for axis and isotropic directions.
"""
import math

import numpy as np
import pytest

import ecmc_workloads as W
import oracle
from test_oracle_threedisk import PASS_CHI2, sample_z

W_CELL = H_CELL = 10.0


def chain(X, Y, n_mem, m, d, ell, reject=True):
    return oracle.run_chain_frame(X, Y, n_mem, m, d[0], d[1], ell, W_CELL, H_CELL,
                                  reject=reject)


def test_accepted_chain_equals_reflecting_rule():
    X, Y, st, rec = chain([1.0, 3.5], [5.0, 5.0], 2, 0, (1.0, 0.0), 2.0)
    X2, Y2, st2, _ = chain([1.0, 3.5], [5.0, 5.0], 2, 0, (1.0, 0.0), 2.0, reject=False)
    assert X.tolist() == [2.5, 4.0] and X.tolist() == X2.tolist()
    assert st.rejected == 0 and st.sum_b == st2.sum_b and st.sum_disp == 2.0


def test_lift_then_wall_is_rejected_and_restored():
    # A lifts B after 1.5; B would need 8 more but the wall is 5.5 away
    X0, Y0 = [1.0, 3.5], [5.0, 5.0]
    X, Y, st, rec = chain(X0, Y0, 2, 0, (1.0, 0.0), 9.5)
    assert X.tolist() == X0 and Y.tolist() == Y0
    assert st.rejected == 1 and st.events == 1 and st.lifts == 1 and st.wall_hits == 1
    assert st.sum_b == 0.0 and st.sum_disp == 0.0
    assert rec["end_id"] == 1  # B was moving when the chain was rejected


def test_frozen_contact_is_rejected_and_restored():
    # member at 1, frozen disk (object 1) at 4 on the same line
    X0, Y0 = [1.0, 4.0], [5.0, 5.0]
    X, Y, st, _ = chain(X0, Y0, 1, 0, (1.0, 0.0), 2.5)
    assert X.tolist() == X0 and st.rejected == 1 and st.frozen_hits == 1 and st.events == 1
    # with a budget that ends before the contact the chain is accepted
    X, Y, st, _ = chain(X0, Y0, 1, 0, (1.0, 0.0), 1.5)
    assert X.tolist() == [2.5, 4.0] and st.rejected == 0


def test_budget_ending_on_the_wall_is_accepted():
    X, Y, st, _ = chain([7.0], [5.0], 1, 0, (1.0, 0.0), 3.0)
    assert X.tolist() == [10.0] and st.rejected == 0 and st.wall_hits == 0


def test_isotropic_chain_rejected_at_wall():
    d = (0.6, 0.8)
    X, Y, st, _ = chain([5.0], [5.0], 1, 0, d, 7.0)  # y would reach 10.6
    assert X.tolist() == [5.0] and Y.tolist() == [5.0] and st.rejected == 1
    X, Y, st, _ = chain([5.0], [5.0], 1, 0, d, 6.0)
    assert st.rejected == 0 and X[0] == 5.0 + 6.0 * 0.6 and Y[0] == 5.0 + 6.0 * 0.8


def chain_sign(seed, t, cell, k):
    v = oracle.philox([t, 1, cell, k], [seed, 0])
    return -1.0 if (v[1] >> 63) else 1.0


@pytest.mark.parametrize("seed", range(8))
def test_one_disk_per_cell_closed_form(seed):
    # 2x2 cells of side 5 without shift, one disk in each, every two disks
    # more than sigma apart in y (periodic images included), so no contact
    # can occur; sweep 0 moves along x, and the disk's chain is accepted iff
    # the budget fits before the wall ahead
    L, ell = 10.0, 1.7
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.2, 4.8, 4)
    v = rng.uniform(0.0, 1.0, 4)
    x = np.array([u[0], 5.0 + u[1], u[2], 5.0 + u[3]])
    y = np.array([0.5, 3.0, 5.5, 8.0]) + v
    p = oracle.make_params(4, L, 1.0, 2, 2, ell, 1, 100 + seed, flags=oracle.FLAG_NO_SHIFT,
                           boundary=oracle.BOUNDARY_REJECT)
    xe = x.copy()
    n_rej = 0
    for i in range(4):
        cell = (int(y[i] // 5.0)) * 2 + int(x[i] // 5.0)
        sgn = chain_sign(100 + seed, 0, cell, 0)
        xr = x[i] - 5.0 * (x[i] >= 5.0)
        fits = (xr + ell <= 5.0) if sgn > 0 else (xr - ell >= 0.0)
        if fits:
            xe[i] = x[i] + sgn * ell
        else:
            n_rej += 1
    xx, yy = x.copy(), y.copy()
    st, _ = oracle.sweeps(p, xx, yy, 0, 1)
    assert st.rejected == n_rej and st.chains == 4
    np.testing.assert_allclose(xx, xe, rtol=0, atol=1e-12)
    for i in range(4):
        if xe[i] == x[i]:
            assert xx[i] == x[i]  # rejected: bitwise unchanged
    assert yy.tolist() == y.tolist()


@pytest.mark.parametrize("dir_mode", [oracle.DIR_PM_AXIS_ALT, oracle.DIR_ISOTROPIC])
def test_budget_beyond_the_cell_rejects_everything(dir_mode):
    N, eta = 256, 0.70
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    p0 = oracle.make_params(N, L, 1.0, 2, 2, 2.0, 4, 5)
    oracle.sweeps(p0, x, y, 0, 20)  # melt with the reflecting rule
    ell = 1.5 * L / 2 * math.sqrt(2.0)  # beyond the cell diagonal
    p = oracle.make_params(N, L, 1.0, 2, 2, ell, 4, 5, dir_mode=dir_mode,
                           boundary=oracle.BOUNDARY_REJECT)
    xx, yy = x.copy(), y.copy()
    st, _ = oracle.sweeps(p, xx, yy, 20, 5)
    assert st.chains == 5 * 4 * 4 and st.rejected == st.chains
    assert st.sum_b == 0.0 and st.sum_disp == 0.0 and st.sum_disp_w == 0.0
    assert xx.tolist() == x.tolist() and yy.tolist() == y.tolist()


@pytest.mark.parametrize("dir_mode", [oracle.DIR_PM_AXIS_ALT, oracle.DIR_ISOTROPIC])
def test_rejection_with_replacement_samples_uniform_measure(dir_mode):
    z, st = sample_z(3.5, 0.6, 4, 200_000, dir_mode=dir_mode, boundary=oracle.BOUNDARY_REJECT)
    assert st.rejected > 0.1 * st.chains and st.rejected < 0.9 * st.chains
    assert np.mean(z**2) < PASS_CHI2 and np.max(np.abs(z)) < 4.5
