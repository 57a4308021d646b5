"""Pins of the per-sweep draws (Sec. 3.4 steps 1-3) and of the binning, in
two and three dimensions.

The Philox words come from numpy's own Philox4x64 (an implementation
independent of the oracle's), the colour orders from itertools' enumeration of
permutations in lexicographic order; the oracle's shift and its decoding of
the permutation number must reproduce both for every sweep.  Then the
statistics the paper asks of the draws: shifts uniform over the cell on every
axis and uncorrelated, every colour equally likely at every position of the
order.  The 3D cell index is compared with exact rational arithmetic.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import ecmc_workloads as W
import oracle

PERMS4 = list(itertools.permutations(range(4)))
PERMS8 = list(itertools.permutations(range(8)))


def numpy_philox(ctr, key):
    # numpy advances the 256-bit counter by one before producing a block
    start = (sum(c << (64 * i) for i, c in enumerate(ctr)) - 1) % 2**256
    words = np.array([(start >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(counter=words, key=np.array(key, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


def unit(u):
    return (u >> 11) / 2.0**53


@pytest.mark.parametrize("seed,replica", [(0, 0), (7, 3), (2**63 + 5, 2**40)])
def test_2d_draws_follow_philox_and_lexicographic_order(seed, replica):
    L = 24.0
    p = oracle.make_params(4, L, 1.0, 4, 6, 1.0, 1, seed, replica)
    for t in (0, 1, 2, 17, 1000, 2**40 + 3):
        u = numpy_philox([t, 0, 0, 0], [seed, replica])
        sx, sy, perm = oracle.sweep_draws(p, t)
        assert sx == unit(u[0]) * (L / 4)
        assert sy == unit(u[1]) * (L / 6)
        assert tuple(perm) == PERMS4[(u[2] * 24) >> 64]


@pytest.mark.parametrize("seed,replica", [(0, 0), (11, 1), (2**64 - 1, 9)])
def test_3d_draws_follow_philox_and_lexicographic_order(seed, replica):
    L = 30.0
    p = oracle.make_params3(8, L, 1.0, 6, 1.0, 1, seed)
    p.replica = replica
    for t in (0, 1, 5, 99, 123456789):
        u = numpy_philox([t, 0, 0, 0], [seed, replica])
        sh, perm = oracle.sweep_draws3(p, t)
        assert sh == [unit(u[a]) * (L / 6) for a in range(3)]
        assert tuple(perm) == PERMS8[(u[3] * 40320) >> 64]


def test_3d_shift_is_uniform_and_uncorrelated():
    L, cells = 20.0, 4
    w = L / cells
    p = oracle.make_params3(8, L, 1.0, cells, 1.0, 1, 5)
    s = np.array([oracle.sweep_draws3(p, t)[0] for t in range(20000)])
    assert np.all((s >= 0) & (s < w))
    for a in range(3):
        hist = np.histogram(s[:, a], bins=20, range=(0, w))[0]
        assert np.sum((hist - 1000.0) ** 2 / 1000.0) < 55.0  # 19 degrees of freedom
    c = np.corrcoef(s.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 0.03)


def test_3d_every_colour_is_equally_likely_at_every_position():
    p = oracle.make_params3(8, 20.0, 1.0, 4, 1.0, 1, 6)
    n = 16000
    counts = np.zeros((8, 8))
    for t in range(n):
        _, perm = oracle.sweep_draws3(p, t)
        counts[np.arange(8), perm] += 1
    assert np.all(counts.sum(axis=1) == n) and np.all(counts.sum(axis=0) == n)
    expect = n / 8.0
    chi2 = np.sum((counts - expect) ** 2 / expect, axis=1)
    assert np.all(chi2 < 27.0)  # 7 degrees of freedom per position, p ~ 3e-4


def test_3d_binning_matches_exact_arithmetic():
    N, eta, cells = 4096, 0.45, 8
    L = W.box_side3(N, eta)
    p = oracle.make_params3(N, L, 1.0, cells, 1.0, 2, 8)
    x, y, z = W.cubic_lattice(N, L)
    oracle.sweeps3(p, x, y, z, 0, 3)
    cell = oracle.bin_cells3(p, 3, x, y, z)
    sh, _ = oracle.sweep_draws3(p, 3)
    w = Fraction(L) / cells
    bad = 0
    for i in range(0, N, 5):
        c = int(cell[i])
        got = (c % cells, (c // cells) % cells, c // (cells * cells))
        for v, s, g in zip((x[i], y[i], z[i]), sh, got):
            u = (Fraction(v) - Fraction(s)) % Fraction(L)
            exact = min(int(u / w), cells - 1)
            if exact != g:
                # only a centre within rounding of a cell wall may differ
                assert abs(float(u - exact * w)) < 1e-12 or abs(float(u - g * w)) < 1e-12
                bad += 1
    assert bad <= 2
    counts = np.bincount(cell, minlength=cells**3)
    assert counts.sum() == N and len(counts) == cells**3


@pytest.mark.parametrize("seed,replica", [(4, 0), (99, 7)])
def test_start_disks_are_drawn_with_replacement_by_the_stated_rule(seed, replica):
    # every chain record's start disk is member floor(v0 n_c / 2^64), in
    # ascending id, of its cell, v0 the first Philox word of (t, 1, c, k)
    N, eta, cells, nm = 1024, 0.70, 4, 6
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, cells, cells, 1.0, nm, seed, replica)
    oracle.sweeps(p, x, y, 0, 2)
    repeats = 0
    for t in (2, 3):
        cell = oracle.bin_cells(p, t, x, y)
        _, recs = oracle.sweeps(p, x, y, t, 1, records=True)
        for c in range(cells * cells):
            members = np.flatnonzero(cell == c)  # ascending id
            starts = []
            for k in range(nm):
                v = numpy_philox([t, 1, c, k], [seed, replica])
                starts.append(int(members[(v[0] * len(members)) >> 64]))
            assert recs[0, c, :]["start_id"].tolist() == starts
            repeats += len(starts) - len(set(starts))
    assert repeats > 0  # 6 draws from about 64 members repeat in about a fifth of the cells
