"""The oracle's g(r) near contact against textbook local Monte Carlo
(tests/localmc.c, Metropolis displacement moves), the reference of the
paper's Fig. 3: N = 100 disks at eta = 0.55, ordered-pair counts in ten
0.05 sigma bins from sigma, batch means on both sides.

  - the PEC sweep with start disks drawn with replacement agrees with local
    Monte Carlo in every bin, for the reflecting and the rejecting rule
    ("PEC-refl" and "PEC-rej" of Fig. 3);
  - shuffled lists of distinct starts (n_m = 10 > 1) distort g(r) right at
    contact, as Fig. 3 (left) shows: the first bin falls many standard errors
    below the reference;
  - the same for the striped decomposition under the rejecting rule (two
    stripes of 50 disks, n_m = 40): with replacement it agrees, shuffled
    lists are biased;
  - the three-dimensional sweep against local Monte Carlo of hard spheres
    (N = 125 at eta = 0.40).
"""
import ctypes as C
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import ecmc_workloads as W
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
N, ETA, R0, DR, NB = 100, 0.55, 1.0, 0.05, 10
NBATCH, PER = 20, 1000


@pytest.fixture(scope="module")
def local_mc():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    d = tempfile.mkdtemp()
    so = os.path.join(d, "localmc.so")
    subprocess.run([gcc, "-O2", "-shared", "-fPIC", os.path.join(HERE, "localmc.c"), "-o", so,
                    "-lm"], check=True)
    lib = C.CDLL(so)
    lib.localmc_run.restype = C.c_longlong
    lib.localmc_run.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                C.c_void_p, C.c_longlong, C.c_uint64, C.c_double, C.c_double,
                                C.c_int, C.c_void_p]
    L = W.box_side(N, ETA)
    x, y = W.square_lattice(N, L)
    lib.localmc_run(N, L, 1.0, 0.15, x.ctypes.data, y.ctypes.data, 2000, 7, R0, DR, NB, None)
    out = []
    acc = 0
    for b in range(NBATCH):
        c = np.zeros(NB, np.int64)
        acc += lib.localmc_run(N, L, 1.0, 0.15, x.ctypes.data, y.ctypes.data, PER, 100 + b, R0,
                               DR, NB, c.ctypes.data)
        out.append(c / PER)
    shutil.rmtree(d, ignore_errors=True)
    assert 0.3 < acc / (NBATCH * PER * N) < 0.8  # a working acceptance rate
    return np.array(out)


def pec_counts(list_mode, boundary=oracle.BOUNDARY_REFLECT):
    # the rejecting rule needs short chains to mix (a third of them are
    # rejected at ell = 0.3) and a longer melt from the lattice
    ell, melt = (1.0, 500) if boundary == oracle.BOUNDARY_REFLECT else (0.3, 2000)
    L = W.box_side(N, ETA)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, 2, 2, ell, 10, 5, list_mode=list_mode, boundary=boundary)
    oracle.sweeps(p, x, y, 0, melt)
    t, out = melt, []
    for _ in range(NBATCH):
        c = np.zeros(NB, np.int64)
        for _ in range(PER):
            oracle.sweeps(p, x, y, t, 1)
            t += 1
            c += oracle.gr_counts(L, x, y, R0, DR, NB)
        out.append(c / PER)
    return np.array(out)


def zscores(a, b):
    se = np.sqrt(a.var(0, ddof=1) / len(a) + b.var(0, ddof=1) / len(b))
    return (b.mean(0) - a.mean(0)) / se


@pytest.mark.parametrize("boundary", [oracle.BOUNDARY_REFLECT, oracle.BOUNDARY_REJECT])
def test_with_replacement_matches_local_monte_carlo(local_mc, boundary):
    z = zscores(local_mc, pec_counts(oracle.LIST_WITH_REPL, boundary))
    assert np.mean(z**2) < 2.5 and np.max(np.abs(z)) < 4.5, z


@pytest.mark.parametrize("boundary", [oracle.BOUNDARY_REFLECT, oracle.BOUNDARY_REJECT])
def test_shuffled_lists_distort_contact_values(local_mc, boundary):
    z = zscores(local_mc, pec_counts(oracle.LIST_WITHOUT_REPL, boundary))
    assert z[0] < -6.0 and np.mean(z**2) > 10.0, z


def stripe_counts(list_mode, nm=40):
    # two stripes of 50 disks: n_m = 40 chains per stripe
    L = W.box_side(N, ETA)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, 2, 2, 1.0, nm, 5, list_mode=list_mode,
                           boundary=oracle.BOUNDARY_REJECT)
    oracle.stripe_sweeps(p, x, y, 0, 500)
    t, out = 500, []
    for _ in range(NBATCH):
        c = np.zeros(NB, np.int64)
        for _ in range(PER):
            oracle.stripe_sweeps(p, x, y, t, 1)
            t += 1
            c += oracle.gr_counts(L, x, y, R0, DR, NB)
        out.append(c / PER)
    return np.array(out)


def test_stripes_with_replacement_match_local_monte_carlo(local_mc):
    z = zscores(local_mc, stripe_counts(oracle.LIST_WITH_REPL))
    assert np.mean(z**2) < 2.5 and np.max(np.abs(z)) < 4.5, z


def test_stripes_with_shuffled_lists_are_biased(local_mc):
    z = zscores(local_mc, stripe_counts(oracle.LIST_WITHOUT_REPL))
    assert np.mean(z**2) > 10.0, z


# -- three dimensions ------------------------------------------------------------
def test_spheres_match_local_monte_carlo():
    # N = 125 spheres at eta = 0.40, 2 x 2 x 2 cells, against localmc3_run
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    n3, eta3, nbatch, per = 125, 0.40, 20, 400
    d = tempfile.mkdtemp()
    so = os.path.join(d, "localmc.so")
    subprocess.run([gcc, "-O2", "-shared", "-fPIC", os.path.join(HERE, "localmc.c"), "-o", so,
                    "-lm"], check=True)
    lib = C.CDLL(so)
    lib.localmc3_run.restype = C.c_longlong
    lib.localmc3_run.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_longlong, C.c_uint64, C.c_double,
                                 C.c_double, C.c_int, C.c_void_p]
    L = W.box_side3(n3, eta3)
    x, y, z = W.cubic_lattice(n3, L)
    lib.localmc3_run(n3, L, 1.0, 0.12, x.ctypes.data, y.ctypes.data, z.ctypes.data, 1500, 7,
                     R0, DR, NB, None)
    lm = []
    for b in range(nbatch):
        c = np.zeros(NB, np.int64)
        lib.localmc3_run(n3, L, 1.0, 0.12, x.ctypes.data, y.ctypes.data, z.ctypes.data, per,
                         100 + b, R0, DR, NB, c.ctypes.data)
        lm.append(c / per)
    shutil.rmtree(d, ignore_errors=True)

    def counts3(x, y, z):
        sep = []
        for a in (x, y, z):
            da = a[None, :] - a[:, None]
            sep.append(da - L * np.floor(da / L + 0.5))
        dd = np.sqrt(sep[0] ** 2 + sep[1] ** 2 + sep[2] ** 2)
        np.fill_diagonal(dd, -1.0)
        return np.histogram(dd.ravel(), bins=NB, range=(R0, R0 + NB * DR))[0]

    x, y, z = W.cubic_lattice(n3, L)
    p3 = oracle.make_params3(n3, L, 1.0, 2, 1.0, 10, 5)
    oracle.sweeps3(p3, x, y, z, 0, 500)
    t, pe = 500, []
    for _ in range(nbatch):
        c = np.zeros(NB, np.int64)
        for _ in range(per):
            oracle.sweeps3(p3, x, y, z, t, 1)
            t += 1
            c += counts3(x, y, z)
        pe.append(c / per)
    zz = zscores(np.array(lm), np.array(pe))
    assert np.mean(zz**2) < 2.5 and np.max(np.abs(zz)) < 4.5, zz
