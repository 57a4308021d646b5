"""Pins of the oracle's striped decomposition (Sec. 3.4, Fig. 3 "stripes":
chains inside stripes that span the box along the chain axis, rejected when
they touch a disk of a neighbouring stripe).

  - closed forms of single chains on hand-built stripe frames: a head-on
    lift, a lift across the periodic end of the stripe, a move backwards
    through it, an offset contact, a frozen contact that rejects the chain
    (or turns it back under the reflecting rule), a lift followed by a
    frozen contact restoring both members, ties, the chain's end before a
    contact at equal distance, and a disk behind that is reached only by
    going round the stripe;
  - one disk per stripe with no contact possible: every chain moves its disk
    by +-ell around the box, the signs recomputed from Philox;
  - invariants of whole sweeps: coordinates across the axis never change,
    no overlap, the stripes of a colour in either order give the same
    trajectory, a run split in two gives the same trajectory;
  - three disks in a periodic box: with replacement the sampled
    pair-distance histogram matches the exact uniform-measure distribution
    (tests/threedisk_exact.py) for both boundary rules; shuffled lists of
    distinct starts do not (the stripes curve of Fig. 3);
  - the pressure at eta = 0.1 against the virial series: the contact value
    of g(r) (eq. pressure) under the rejecting rule, the member-weighted
    collision estimator under the reflecting rule.
"""
import math

import numpy as np
import pytest

import ecmc_workloads as W
import oracle
import threedisk_exact as T
from bench import contact_value
from test_oracle_gcontact import virial_golden
from test_oracle_threedisk import FAIL_CHI2, NBATCH, PASS_CHI2, edges_for

L10 = 10.0
REJECT_, REFLECT_ = oracle.BOUNDARY_REJECT, oracle.BOUNDARY_REFLECT


def chain(U, V, n_mem, m, sign, ell, reject=True, keys=None):
    return oracle.run_chain_stripe(U, V, n_mem, m, sign, ell, L10, keys=keys, reject=reject)


# -- single chains -----------------------------------------------------------
def test_head_on_lift():
    U, st, rec, rej = chain([1.0, 3.5], [0.5, 0.5], 2, 0, 1, 2.0)
    assert U.tolist() == [2.5, 4.0] and not rej
    assert st.lifts == 1 and st.events == 1 and st.sum_b == 1.0 and rec["end_id"] == 1


def test_lift_across_the_periodic_end():
    # disk 1 is 1.25 ahead of disk 0 round the end of the stripe at L = 10
    U, st, rec, rej = chain([9.5, 0.75], [0.0, 0.0], 2, 0, 1, 1.25)
    assert U.tolist() == [9.75, 1.75] and st.lifts == 1 and st.sum_b == 1.0


def test_backwards_through_the_periodic_end():
    U, st, _, _ = chain([0.25], [0.0], 1, 0, -1, 0.5)
    assert U.tolist() == [9.75] and st.events == 0


def test_offset_contact():
    # across offset 0.6: contact after 3 - 0.8 = 2.2, separation 0.8 along
    U, st, _, _ = chain([1.0, 4.0], [0.0, 0.6], 2, 0, 1, 5.0)
    assert U == pytest.approx([3.2, 6.8], abs=1e-14)
    assert st.sum_b == pytest.approx(0.8, abs=1e-15)


def test_frozen_contact_rejects_the_chain():
    U0, V = [1.0, 3.0], [0.0, 0.5]
    U, st, _, rej = chain(U0, V, 1, 0, 1, 2.0)  # contact after 2 - sqrt(0.75) < 2
    assert rej and U.tolist() == U0
    assert st.rejected == 1 and st.frozen_hits == 1 and st.sum_b == 0.0
    U, st, _, rej = chain(U0, V, 1, 0, 1, 1.0)  # the budget ends first
    assert not rej and U.tolist() == [2.0, 3.0] and st.rejected == 0


def test_lift_then_frozen_contact_restores_both_members():
    U0, V = [1.0, 2.5, 5.0], [0.0, 0.0, 0.0]
    U, st, rec, rej = chain(U0, V, 2, 0, 1, 3.0)
    assert rej and U.tolist() == U0
    assert st.events == 2 and st.lifts == 1 and st.frozen_hits == 1 and st.sum_b == 0.0
    assert rec["end_id"] == 1


def test_reflecting_rule_turns_back_at_a_frozen_disk():
    # 0.5 to the lift, 1.5 to the frozen disk, then 1.0 back
    U, st, _, rej = chain([1.0, 2.5, 5.0], [0.0, 0.0, 0.0], 2, 0, 1, 3.0, reject=False)
    assert not rej and U.tolist() == [1.5, 3.0, 5.0]
    assert st.lifts == 1 and st.frozen_hits == 1 and st.sum_b == 2.0


def test_equal_travel_goes_to_the_smaller_key():
    U, st, _, _ = chain([0.0, 2.0, 2.0], [0.0, 0.6, -0.6], 3, 0, 1, 1.5, keys=[0, 5, 3])
    assert U[1] == 2.0 and U[2] == pytest.approx(2.3, abs=1e-14) and st.lifts == 1


def test_chain_end_before_contact_at_equal_distance():
    U, st, _, _ = chain([0.0, 2.0], [0.0, 0.0], 2, 0, 1, 1.0)
    assert U.tolist() == [1.0, 2.0] and st.events == 0


def test_disk_behind_is_reached_only_round_the_stripe():
    U, st, _, _ = chain([5.0, 4.0], [0.0, 0.0], 2, 0, 1, 3.0)
    assert U.tolist() == [8.0, 4.0] and st.events == 0
    U, st, _, _ = chain([5.0, 4.0], [0.0, 0.0], 2, 0, 1, 9.0)
    assert U.tolist() == [3.0, 5.0] and st.lifts == 1


# -- whole sweeps ------------------------------------------------------------
@pytest.mark.parametrize("t", [0, 1, 2, 7, 40])
@pytest.mark.parametrize("boundary", [oracle.BOUNDARY_REJECT, oracle.BOUNDARY_REFLECT])
def test_one_disk_per_stripe_moves_by_the_drawn_signs(t, boundary):
    # the diagonal holds one disk per stripe for either axis, and stripes
    # 2 apart keep every pair out of contact
    L, S, ell, nm = 8.0, 4, 0.75, 3
    x0 = np.array([1.0, 3.0, 5.0, 7.0])
    x, y = x0.copy(), x0.copy()
    p = oracle.make_params(4, L, 1.0, S, S, ell, nm, 9, 2, flags=oracle.FLAG_NO_SHIFT,
                           boundary=boundary)
    st, recs = oracle.stripe_sweeps(p, x, y, t, 1, records=True)
    along, across = (y, x) if t & 1 else (x, y)
    assert across.tolist() == x0.tolist()
    for i in range(4):
        k = i  # disk i sits in stripe i
        u = x0[i]
        for c in range(nm):
            v = oracle.philox([t, 1, k, c], [9, 2])
            u = (u + (-ell if v[1] >> 63 else ell)) % L
        assert along[i] == u
        assert recs[0, k, :]["start_id"].tolist() == [i] * nm
    assert st.events == 0 and st.chains == 4 * nm and st.rejected == 0


def dense(N=1024, eta=0.70, S=8, ell=1.3, nm=8, boundary=oracle.BOUNDARY_REJECT, flags=0):
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, S, S, ell, nm, 5, flags=flags, boundary=boundary)
    return p, x, y, L


@pytest.mark.parametrize("boundary", [oracle.BOUNDARY_REJECT, oracle.BOUNDARY_REFLECT])
def test_dense_sweeps_keep_disks_apart_and_in_their_stripes(boundary):
    p, x, y, L = dense(boundary=boundary)
    tot = oracle.Stats()
    for t in range(12):
        across = (x if t & 1 else y).copy()
        oracle.stripe_sweeps(p, x, y, t, 1, stats=tot)
        assert (x if t & 1 else y).tolist() == across.tolist()
    assert oracle.min_dist2(L, x, y) >= 1.0 - 1e-12
    assert tot.events > 10 * tot.chains and tot.lifts > 0 and tot.frozen_hits > 0
    assert tot.wall_hits == 0
    if boundary == oracle.BOUNDARY_REJECT:
        assert 0 < tot.rejected < tot.chains
    else:
        assert tot.rejected == 0


def test_order_of_stripes_within_a_colour_is_irrelevant():
    p, x, y, L = dense()
    q, u, v, _ = dense(flags=oracle.FLAG_REVERSE_CELLS)
    sa, _ = oracle.stripe_sweeps(p, x, y, 0, 8)
    sb, _ = oracle.stripe_sweeps(q, u, v, 0, 8)
    assert x.tolist() == u.tolist() and y.tolist() == v.tolist()
    assert sa.events == sb.events and sa.rejected == sb.rejected


def test_split_run_is_bitwise_identical():
    p, x, y, L = dense(boundary=oracle.BOUNDARY_REFLECT)
    q, u, v, _ = dense(boundary=oracle.BOUNDARY_REFLECT)
    oracle.stripe_sweeps(p, x, y, 0, 9)
    oracle.stripe_sweeps(q, u, v, 0, 4)
    oracle.stripe_sweeps(q, u, v, 4, 5)
    assert x.tolist() == u.tolist() and y.tolist() == v.tolist()


def test_invalid_parameters_are_refused():
    L = 10.0
    for kw in ({"cells_x": 3}, {"cells_x": 12}, {"dir_mode": oracle.DIR_ISOTROPIC}):
        args = dict(cells_x=4, dir_mode=oracle.DIR_PM_AXIS_ALT)
        args.update(kw)
        p = oracle.make_params(4, L, 1.0, args["cells_x"], 4, 1.0, 1, 1,
                               dir_mode=args["dir_mode"])
        with pytest.raises(ValueError):
            oracle.stripe_sweeps(p, np.zeros(4), np.zeros(4), 0, 1)


# -- three disks: the uniform measure ------------------------------------------
def stripe_z(L, ell, nm, n_sweeps, list_mode=oracle.LIST_WITH_REPL,
             boundary=oracle.BOUNDARY_REJECT, seed=7):
    x = np.array([0.3, 1.6, 2.9])
    y = np.array([0.4, 2.2, 1.0])
    p = oracle.make_params(3, L, 1.0, 2, 2, ell, nm, seed, 0, list_mode=list_mode,
                           boundary=boundary)
    oracle.stripe_sweeps(p, x, y, 0, 100)
    st = oracle.Stats()
    sx = np.empty((n_sweeps, 3))
    sy = np.empty((n_sweeps, 3))
    for s in range(n_sweeps):
        oracle.stripe_sweeps(p, x, y, 100 + s, 1, stats=st)
        sx[s], sy[s] = x, y

    def md(i, j):
        dx = sx[:, i] - sx[:, j]
        dy = sy[:, i] - sy[:, j]
        dx -= L * np.round(dx / L)
        dy -= L * np.round(dy / L)
        return np.hypot(dx, dy)

    d = np.stack([md(0, 1), md(0, 2), md(1, 2)], 1)
    e = edges_for(L)
    pex = T.bin_probabilities(e, L, 1.0)
    hb = np.array([np.histogram(b.ravel(), e)[0] for b in np.array_split(d, NBATCH)], float)
    fr = hb / hb.sum(1, keepdims=True)
    se = fr.std(0, ddof=1) / math.sqrt(NBATCH)
    return (fr.mean(0) - pex) / se, st


@pytest.mark.parametrize("boundary", [oracle.BOUNDARY_REJECT, oracle.BOUNDARY_REFLECT])
@pytest.mark.parametrize("L,ell,nm", [(3.5, 3.0, 4), (3.8, 5.0, 8)])
def test_with_replacement_samples_uniform_measure(L, ell, nm, boundary):
    z, st = stripe_z(L, ell, nm, 200_000, boundary=boundary)
    assert st.frozen_hits > 0 and st.lifts > 0
    assert np.mean(z**2) < PASS_CHI2 and np.max(np.abs(z)) < 4.5


@pytest.mark.parametrize("boundary,L,ell,nm", [(oracle.BOUNDARY_REJECT, 3.5, 3.0, 4),
                                               (oracle.BOUNDARY_REFLECT, 3.8, 5.0, 8)])
def test_shuffled_lists_are_biased(boundary, L, ell, nm):
    z, _ = stripe_z(L, ell, nm, 400_000, list_mode=oracle.LIST_WITHOUT_REPL, boundary=boundary)
    assert np.mean(z**2) > FAIL_CHI2


# -- pressure at low density ---------------------------------------------------
@pytest.mark.parametrize("boundary", [oracle.BOUNDARY_REJECT, oracle.BOUNDARY_REFLECT])
def test_low_density_pressure_matches_virial_series(boundary):
    N, eta, S, dr, nb = 400, 0.10, 10, 0.01, 20
    L = W.box_side(N, eta)
    rho = N / L**2
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, S, S, 2.0, 10, 3, boundary=boundary)
    oracle.stripe_sweeps(p, x, y, 0, 200)
    t, via_g, via_chain = 200, [], []
    for _ in range(10):
        counts = np.zeros(nb, np.int64)
        st = oracle.Stats()
        for _ in range(400):
            oracle.stripe_sweeps(p, x, y, t, 1, stats=st)
            t += 1
            counts += oracle.gr_counts(L, x, y, 1.0, dr, nb)
        R, g = oracle.gr_normalise(counts.astype(float), 400, N, L, 1.0, dr)
        via_g.append(1.0 + 0.5 * math.pi * rho * contact_value(R, g))
        via_chain.append(1.0 + st.sum_b_w / st.sum_disp_w)
    gv = virial_golden()
    x2 = 0.5 * math.pi * rho
    vir = 1.0 + x2 + gv["B3_over_B2sq"] * x2**2 + gv["B4_over_B2cu"] * x2**3
    # the collision estimator holds for the reflecting rule only; the
    # rejecting rule's pressure comes from the contact value of g(r)
    v = np.array(via_chain if boundary == oracle.BOUNDARY_REFLECT else via_g)
    z, se = v.mean(), v.std(ddof=1) / math.sqrt(len(v))
    assert abs(z - vir) < 4.0 * se + 1e-3, (z, vir, se)


@pytest.mark.parametrize("boundary", [REJECT_, REFLECT_])
def test_stripe_chains_never_carry_a_disk_through_another(boundary):
    from test_oracle_invariants import cyclic_orders_kept

    p, x, y, L = dense(boundary=boundary, ell=3.0)
    oracle.stripe_sweeps(p, x, y, 0, 4)
    for t in range(4, 10):
        x0, y0 = x.copy(), y.copy()
        oracle.stripe_sweeps(p, x, y, t, 1)
        along0, along1, across = (x0, x, y0) if t % 2 == 0 else (y0, y, x0)
        ok, checked = cyclic_orders_kept(along0, along1, across, L)
        assert ok, "a disk passed through another in sweep %d" % t
        assert checked > 10
