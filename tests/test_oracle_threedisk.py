"""Pin (b): three hard disks in a small periodic box, 2x2 cells.

The pair-distance histogram sampled by the oracle's sweep must match the
exact distribution of the uniform measure on non-overlapping configurations
(numerical integration, tests/threedisk_exact.py), which is itself checked
against direct rejection sampling.  Chains started with replacement (Sec. 3.4
step 5) pass; the shuffled list of distinct starts, the "+ only" direction
rule and axis chains reflected specularly at frozen disks do not (Sec. 3.4,
Fig. 2, and the discussion of detailed balance in Sec. 3.2)."""
import math

import numpy as np
import pytest

import oracle
import threedisk_exact as T

NBIN = 14
NBATCH = 50


def edges_for(L):
    return np.linspace(1.0, L / math.sqrt(2.0), NBIN + 1)


def test_exact_distribution_matches_rejection_sampling():
    L = 3.5
    e = edges_for(L)
    p = T.bin_probabilities(e, L, 1.0)
    rng = np.random.default_rng(2024)
    P = rng.random((1_500_000, 3, 2)) * L

    def md(a, b):
        d = a - b
        d -= L * np.round(d / L)
        return np.hypot(d[:, 0], d[:, 1])

    d12, d13, d23 = md(P[:, 0], P[:, 1]), md(P[:, 0], P[:, 2]), md(P[:, 1], P[:, 2])
    ok = (d12 >= 1.0) & (d13 >= 1.0) & (d23 >= 1.0)
    n = int(ok.sum())
    h = np.histogram(np.concatenate([d12[ok], d13[ok], d23[ok]]), e)[0] / (3.0 * n)
    # the three pair distances of one sample are dependent: allow 5 sigma of a
    # per-pair binomial with 3n/... samples (conservative: n samples)
    z = (h - p) / np.sqrt(p * (1 - p) / n)
    assert np.max(np.abs(z)) < 5.0
    assert abs(p.sum() - 1.0) < 1e-12


def sample_z(L, ell, nm, n_sweeps, list_mode=oracle.LIST_WITH_REPL,
             dir_mode=oracle.DIR_PM_AXIS_ALT, flags=0, seed=7, boundary=oracle.BOUNDARY_REFLECT):
    x = np.array([0.3, 1.6, 2.9])
    y = np.array([0.4, 2.2, 1.0])
    p = oracle.make_params(3, L, 1.0, 2, 2, ell, nm, seed, 0, dir_mode=dir_mode,
                           list_mode=list_mode, flags=flags, boundary=boundary)
    oracle.sweeps(p, x, y, 0, 100)
    st, sx, sy = oracle.sweeps_snap(p, x, y, 100, n_sweeps)

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
    z = (fr.mean(0) - pex) / se
    return z, st


# chi^2 per bin of batch-mean z scores: about 1 for a correct sampler
PASS_CHI2 = 2.5
FAIL_CHI2 = 4.0


@pytest.mark.parametrize("L,ell,nm", [(3.5, 3.0, 4), (3.8, 5.0, 8)])
def test_with_replacement_samples_uniform_measure(L, ell, nm):
    z, st = sample_z(L, ell, nm, 200_000)
    assert st.events > 100_000 and st.frozen_hits > 0 and st.wall_hits > 0
    assert np.mean(z**2) < PASS_CHI2 and np.max(np.abs(z)) < 4.5


def test_isotropic_specular_samples_uniform_measure():
    z, st = sample_z(3.5, 3.0, 4, 200_000, dir_mode=oracle.DIR_ISOTROPIC)
    assert np.mean(z**2) < PASS_CHI2 and np.max(np.abs(z)) < 4.5


def test_without_replacement_is_biased():
    z, _ = sample_z(3.8, 5.0, 8, 400_000, list_mode=oracle.LIST_WITHOUT_REPL)
    assert np.mean(z**2) > FAIL_CHI2


def test_positive_only_direction_is_biased():
    z, _ = sample_z(3.5, 3.0, 4, 100_000, dir_mode=oracle.DIR_POS_ONLY)
    assert np.mean(z**2) > FAIL_CHI2 * 10


def test_axis_chains_with_specular_frozen_reflection_are_biased():
    z, _ = sample_z(3.5, 3.0, 4, 100_000, flags=oracle.FLAG_SPECULAR_AXIS)
    assert np.mean(z**2) > FAIL_CHI2 * 10
