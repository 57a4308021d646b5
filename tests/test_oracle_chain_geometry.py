"""Closed-form pins of one event chain in a cell frame (Sec. 3.2 and the
boundary rule of Sec. 3.4, Fig. 1).  Frames are built by hand: the cell is
[0,w] x [0,h], objects 0..n_mem-1 are its members, the rest are frozen."""
import math

import numpy as np
import pytest

import oracle

W = H = 10.0


def chain(X, Y, n_mem, m, d, ell, specular=False, ids=None, imgs=None):
    return oracle.run_chain_frame(X, Y, n_mem, m, d[0], d[1], ell, W, H, ids=ids, imgs=imgs,
                                  specular=specular)


def test_head_on_lift():
    # A moves 1.5 to contact (centres sigma apart), B takes the remaining 0.5
    X, Y, st, rec = chain([1.0, 3.5], [5.0, 5.0], 2, 0, (1.0, 0.0), 2.0)
    assert X.tolist() == [2.5, 4.0] and Y.tolist() == [5.0, 5.0]
    assert st.events == 1 and st.lifts == 1 and rec["end_id"] == 1
    assert st.sum_b == pytest.approx(1.0, abs=1e-15)  # separation along d at contact


def test_offset_contact_distance():
    # impact parameter c = 0.6: contact after b - sqrt(sigma^2 - c^2) = 3 - 0.8
    X, Y, st, rec = chain([1.0, 4.0], [5.0, 5.6], 2, 0, (1.0, 0.0), 3.0)
    assert X[0] == pytest.approx(3.2, abs=1e-14) and X[1] == pytest.approx(4.8, abs=1e-14)
    assert st.sum_b == pytest.approx(0.8, abs=1e-14)
    # the contact puts the two centres exactly sigma apart
    assert math.hypot(4.0 - X[0], 0.6) == pytest.approx(1.0, abs=1e-14)


def test_negative_direction_and_y_axis():
    X, Y, st, _ = chain([5.0, 5.3], [6.0, 3.0], 2, 0, (0.0, -1.0), 2.5)
    # c = 0.3, s = 3 - sqrt(1 - 0.09)
    s = 3.0 - math.sqrt(1.0 - 0.09)
    assert Y[0] == pytest.approx(6.0 - s, abs=1e-14)
    assert Y[1] == pytest.approx(3.0 - (2.5 - s), abs=1e-14)


def test_passing_beside_and_behind_are_not_hit():
    # |c| = 1.0 is not a hit (strict), and a disk behind is never hit
    X, Y, st, _ = chain([1.0, 3.0, 0.5], [5.0, 6.0, 5.0], 3, 0, (1.0, 0.0), 2.0)
    assert st.events == 0 and X[0] == 3.0 and X[2] == 0.5


def test_budget_ends_exactly_at_contact_does_not_lift():
    # the chain end wins a tie with a contact
    X, Y, st, rec = chain([1.0, 3.0], [5.0, 5.0], 2, 0, (1.0, 0.0), 1.0)
    assert X.tolist() == [2.0, 3.0] and st.events == 0 and rec["end_id"] == 0


def test_wall_reflection_axis_chain():
    X, Y, st, _ = chain([9.0], [5.0], 1, 0, (1.0, 0.0), 3.0)
    assert X[0] == 8.0 and st.wall_hits == 1
    X, Y, st, _ = chain([0.5], [5.0], 1, 0, (-1.0, 0.0), 12.0)
    # 0.5 to the left wall, 10 across, 1.5 back from the right wall
    assert X[0] == pytest.approx(8.5, abs=1e-14) and st.wall_hits == 2


def test_contact_beats_wall_on_tie():
    # frozen disk whose contact point coincides with the wall
    X, Y, st, _ = chain([9.0, 11.0], [5.0, 5.0], 1, 0, (1.0, 0.0), 1.5)
    assert st.frozen_hits == 1 and st.wall_hits == 0


def test_axis_chain_turns_back_at_frozen_disk():
    # frozen disk off-centre (c = 0.6); the axis chain reverses at contact
    X, Y, st, _ = chain([8.0, 10.4], [5.0, 5.6], 1, 0, (1.0, 0.0), 2.0)
    s = 2.4 - 0.8
    assert X[0] == pytest.approx(8.0 + s - (2.0 - s), abs=1e-14)
    assert X[1] == 10.4 and st.frozen_hits == 1 and st.events == 1
    assert st.sum_b == pytest.approx(0.8, abs=1e-14)


def test_specular_reflection_at_45_degrees():
    # contact normal at 45 degrees: +x becomes -y (frozen disk above right)
    a = 1.0 / math.sqrt(2.0)
    X, Y, st, _ = chain([5.0, 7.0 + a], [5.0, 5.0 + a], 1, 0, (1.0, 0.0), 3.0, specular=True)
    # moves 2 to contact at (7, 5), then 1 along -y
    assert X[0] == pytest.approx(7.0, abs=1e-13) and Y[0] == pytest.approx(4.0, abs=1e-13)
    # and a frozen disk below right turns +x into +y
    X, Y, st, _ = chain([5.0, 7.0 + a], [5.0, 5.0 - a], 1, 0, (1.0, 0.0), 3.0, specular=True)
    assert X[0] == pytest.approx(7.0, abs=1e-13) and Y[0] == pytest.approx(6.0, abs=1e-13)


def test_corner_reflects_both_components():
    a = 1.0 / math.sqrt(2.0)  # equal components: both walls at the same distance
    X, Y, st, _ = chain([9.5], [9.5], 1, 0, (a, a), 1.0, specular=True)
    s = 0.5 / a
    assert X[0] == pytest.approx(10.0 - (1.0 - s) * a, abs=1e-14)
    assert Y[0] == X[0] and st.wall_hits == 1


def test_equal_distance_tie_takes_smaller_key():
    # two members hit at the same travel distance: the smaller id takes the lift
    X, Y, st, rec = chain([1.0, 3.0, 3.0], [5.0, 5.6, 4.4], 3, 0, (1.0, 0.0), 2.0,
                          ids=[10, 12, 11])
    assert rec["end_id"] == 11
    X, Y, st, rec = chain([1.0, 3.0, 3.0], [5.0, 5.6, 4.4], 3, 0, (1.0, 0.0), 2.0,
                          ids=[10, 11, 12])
    assert rec["end_id"] == 11


def test_overlapping_pair_lifts_with_zero_travel():
    # a pair already closer than sigma: the hit distance is clamped at zero
    X, Y, st, rec = chain([1.0, 1.9], [5.0, 5.0], 2, 0, (1.0, 0.0), 0.5)
    assert X[0] == 1.0 and X[1] == pytest.approx(2.4) and st.events == 1
