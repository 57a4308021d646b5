"""Python access to the oracle: the plain sequential FP64 C implementation of
the parallel event-chain sweep (Kampmann, Boltz, Kierfeld, arXiv:1409.6948).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module; the product library never does.
Everything here is argument marshalling around ``liboracle.so``; the
arithmetic is in ``ecmc_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

DIR_PM_AXIS_ALT = 0
DIR_POS_ONLY = 1
DIR_ISOTROPIC = 2
LIST_WITH_REPL = 0
LIST_WITHOUT_REPL = 1
FLAG_NO_SHIFT = 1
FLAG_BRUTE_FROZEN = 2
FLAG_REVERSE_CELLS = 4
FLAG_FIXED_COLOURS = 8
FLAG_SPECULAR_AXIS = 16
BOUNDARY_REFLECT = 0
BOUNDARY_REJECT = 1


class Params(C.Structure):
    _fields_ = [("N", C.c_int64), ("L", C.c_double), ("sigma", C.c_double),
                ("cells_x", C.c_int), ("cells_y", C.c_int), ("ell", C.c_double),
                ("n_m", C.c_int), ("seed", C.c_uint64), ("replica", C.c_uint64),
                ("dir_mode", C.c_int), ("list_mode", C.c_int), ("flags", C.c_uint),
                ("boundary", C.c_int)]


class Params3(C.Structure):
    _fields_ = [("N", C.c_int64), ("L", C.c_double), ("sigma", C.c_double),
                ("cells", C.c_int), ("ell", C.c_double), ("n_m", C.c_int),
                ("seed", C.c_uint64), ("replica", C.c_uint64), ("flags", C.c_uint)]


class Stats(C.Structure):
    _fields_ = [("sweeps", C.c_int64), ("chains", C.c_int64), ("events", C.c_int64),
                ("lifts", C.c_int64), ("frozen_hits", C.c_int64), ("wall_hits", C.c_int64),
                ("capped", C.c_int64), ("sum_b", C.c_double), ("sum_disp", C.c_double),
                ("sum_b_w", C.c_double), ("sum_disp_w", C.c_double), ("rejected", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


CHAIN_REC = np.dtype([("start_id", np.int64), ("end_id", np.int64), ("events", np.int64),
                      ("walls", np.int64)])

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        d, i64, u64 = C.POINTER(C.c_double), C.c_int64, C.c_uint64
        L.orc_philox4x64_10.argtypes = [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                        C.POINTER(C.c_uint64)]
        L.orc_philox4x64_10.restype = None
        L.orc_sweep_draws.argtypes = [C.POINTER(Params), i64, d, d, C.POINTER(C.c_int)]
        L.orc_sweep_draws.restype = None
        L.orc_bin.argtypes = [C.POINTER(Params), i64, d, d, C.POINTER(C.c_int32)]
        L.orc_bin.restype = C.c_int
        L.orc_default_nm.argtypes = [i64, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double]
        L.orc_default_nm.restype = C.c_int
        L.orc_sweeps.argtypes = [C.POINTER(Params), d, d, i64, i64, C.POINTER(Stats), C.c_void_p]
        L.orc_sweeps.restype = C.c_int
        L.orc_seq_sweeps.argtypes = [i64, C.c_double, C.c_double, C.c_double, i64, u64, u64,
                                     d, d, i64, i64, C.POINTER(Stats)]
        L.orc_seq_sweeps.restype = C.c_int
        L.orc_gr_counts.argtypes = [i64, C.c_double, d, d, C.c_double, C.c_double, C.c_int,
                                    i64, i64, C.POINTER(C.c_int64)]
        L.orc_gr_counts.restype = None
        L.orc_gr_counts_cells.argtypes = [i64, C.c_double, d, d, C.c_double, C.c_double,
                                          C.c_int, C.POINTER(C.c_int64)]
        L.orc_gr_counts_cells.restype = None
        L.orc_suggest_parameters.argtypes = [i64, C.c_double, C.c_double, C.c_double,
                                             C.POINTER(C.c_int), C.POINTER(C.c_double),
                                             C.POINTER(C.c_int)]
        L.orc_suggest_parameters.restype = C.c_int
        L.orc_autocorrelation_time.argtypes = [d, d, i64, C.c_int, i64, C.POINTER(C.c_double),
                                               C.c_void_p]
        L.orc_autocorrelation_time.restype = C.c_int
        L.orc_min_dist2.argtypes = [i64, C.c_double, d, d, C.c_double]
        L.orc_min_dist2.restype = C.c_double
        L.orc_run_chain_frame.argtypes = [C.c_int, C.c_int, d, d, C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int32), C.c_double, C.c_double,
                                          C.c_double, C.c_int, C.c_double, C.c_double,
                                          C.c_double, C.c_int, C.POINTER(Stats), C.c_void_p]
        L.orc_run_chain_frame.restype = C.c_int
        L.orc_sweeps_snap.argtypes = [C.POINTER(Params), d, d, i64, i64, C.POINTER(Stats), d, d]
        L.orc_sweeps_snap.restype = C.c_int
        L.orc_hexatic.argtypes = [i64, C.c_double, d, d, C.c_double, C.c_void_p, C.c_void_p,
                                  C.c_void_p]
        L.orc_hexatic.restype = C.c_int
        P3 = C.POINTER(Params3)
        L.orc3_sweep_draws.argtypes = [P3, i64, d, C.POINTER(C.c_int)]
        L.orc3_sweep_draws.restype = None
        L.orc3_bin.argtypes = [P3, i64, d, d, d, C.POINTER(C.c_int32)]
        L.orc3_bin.restype = C.c_int
        L.orc3_sweeps.argtypes = [P3, d, d, d, i64, i64, C.POINTER(Stats), C.c_void_p]
        L.orc3_sweeps.restype = C.c_int
        L.orc3_run_chain_frame.argtypes = [C.c_int, C.c_int, d, d, d, C.POINTER(C.c_int64),
                                           C.POINTER(C.c_int32), C.c_double, C.c_double,
                                           C.c_int, C.c_int, C.c_int, C.c_double,
                                           C.POINTER(Stats), C.c_void_p]
        L.orc3_run_chain_frame.restype = C.c_int
        L.orc3_min_dist2.argtypes = [i64, C.c_double, d, d, d, C.c_double]
        L.orc3_min_dist2.restype = C.c_double
        L.orc_stripe_draws.argtypes = [C.POINTER(Params), i64, d, C.POINTER(C.c_int)]
        L.orc_stripe_draws.restype = None
        L.orc_stripe_bin.argtypes = [C.POINTER(Params), i64, d, d, C.POINTER(C.c_int32)]
        L.orc_stripe_bin.restype = C.c_int
        L.orc_stripe_sweeps.argtypes = [C.POINTER(Params), d, d, i64, i64, C.POINTER(Stats),
                                        C.c_void_p]
        L.orc_stripe_sweeps.restype = C.c_int
        L.orc_run_chain_stripe.argtypes = [C.c_int, C.c_int, d, d, C.POINTER(C.c_int64),
                                           C.c_double, C.c_double, C.c_int, C.c_int,
                                           C.c_double, C.c_int, C.POINTER(Stats), C.c_void_p]
        L.orc_run_chain_stripe.restype = C.c_int
        _lib = L
    return _lib


def _dptr(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def philox(ctr, key):
    c = (C.c_uint64 * 4)(*[int(v) & (2**64 - 1) for v in ctr])
    k = (C.c_uint64 * 2)(*[int(v) & (2**64 - 1) for v in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(v) for v in o]


def make_params(N, L, sigma, cells_x, cells_y, ell, n_m, seed, replica=0,
                dir_mode=DIR_PM_AXIS_ALT, list_mode=LIST_WITH_REPL, flags=0,
                boundary=BOUNDARY_REFLECT):
    return Params(int(N), float(L), float(sigma), int(cells_x), int(cells_y), float(ell),
                  int(n_m), int(seed), int(replica), int(dir_mode), int(list_mode), int(flags),
                  int(boundary))


def sweep_draws(p, t):
    sx, sy = C.c_double(), C.c_double()
    perm = (C.c_int * 4)()
    lib().orc_sweep_draws(C.byref(p), int(t), C.byref(sx), C.byref(sy), perm)
    return sx.value, sy.value, list(perm)


def bin_cells(p, t, x, y):
    cell = np.empty(p.N, np.int32)
    lib().orc_bin(C.byref(p), int(t), _dptr(x), _dptr(y),
                  cell.ctypes.data_as(C.POINTER(C.c_int32)))
    return cell


def default_nm(N, L, sigma, cells_x, cells_y, ell):
    return lib().orc_default_nm(int(N), float(L), float(sigma), int(cells_x), int(cells_y),
                                float(ell))


def suggest_parameters(N, L, sigma=1.0, min_cell_side=0.0):
    """The closing strategy of Sec. 4: (cells per side, ell, n_m)."""
    c, ell, nm = C.c_int(), C.c_double(), C.c_int()
    rc = lib().orc_suggest_parameters(int(N), float(L), float(sigma), float(min_cell_side),
                                      C.byref(c), C.byref(ell), C.byref(nm))
    if rc != 0:
        raise ValueError("no grid of 2x2 cells fits (rc=%d)" % rc)
    return c.value, ell.value, nm.value


def autocorrelation_time(psi_series, max_lag):
    """tau (eq. tau) and C(0..max_lag) of one complex series [n] or of R
    series [n, R] (replicas, averaged)."""
    z = np.asarray(psi_series, dtype=complex)
    if z.ndim == 1:
        z = z[:, None]
    n, R = z.shape
    re = np.ascontiguousarray(z.real.T)   # series-major for the oracle
    im = np.ascontiguousarray(z.imag.T)
    c = np.empty(int(max_lag) + 1)
    tau = C.c_double()
    rc = lib().orc_autocorrelation_time(_dptr(re), _dptr(im), int(n), int(R), int(max_lag),
                                        C.byref(tau), c.ctypes.data_as(C.c_void_p))
    if rc != 0:
        raise ValueError("bad series (rc=%d)" % rc)
    return tau.value, c


def sweeps(p, x, y, t0, n_sweeps, stats=None, records=False):
    """Run n_sweeps sweeps in place on x, y (float64, id order).  Returns
    (stats, records) where records is a structured array
    [n_sweeps, cells, n_m] of CHAIN_REC or None."""
    st = stats if stats is not None else Stats()
    recs = None
    rp = None
    if records:
        recs = np.zeros((n_sweeps, p.cells_x * p.cells_y, p.n_m), CHAIN_REC)
        rp = recs.ctypes.data_as(C.c_void_p)
    rc = lib().orc_sweeps(C.byref(p), _dptr(x), _dptr(y), int(t0), int(n_sweeps), C.byref(st), rp)
    if rc != 0:
        raise ValueError("oracle rejected the parameters (rc=%d)" % rc)
    return st, recs


def sweeps_snap(p, x, y, t0, n_sweeps, stats=None):
    """Like sweeps(); also returns the configuration after every sweep as
    arrays [n_sweeps, N]."""
    st = stats if stats is not None else Stats()
    sx = np.empty((n_sweeps, p.N))
    sy = np.empty((n_sweeps, p.N))
    rc = lib().orc_sweeps_snap(C.byref(p), _dptr(x), _dptr(y), int(t0), int(n_sweeps),
                               C.byref(st), _dptr(sx), _dptr(sy))
    if rc != 0:
        raise ValueError("oracle rejected the parameters (rc=%d)" % rc)
    return st, sx, sy


def seq_sweeps(N, L, sigma, ell, n_chains, seed, replica, x, y, t0, n_sweeps, stats=None):
    st = stats if stats is not None else Stats()
    rc = lib().orc_seq_sweeps(int(N), float(L), float(sigma), float(ell), int(n_chains),
                              int(seed), int(replica), _dptr(x), _dptr(y), int(t0),
                              int(n_sweeps), C.byref(st))
    if rc != 0:
        raise ValueError("oracle rejected the parameters (rc=%d)" % rc)
    return st


def gr_counts(L, x, y, sigma, dr, nbins, i_begin=0, i_end=None, counts=None):
    N = x.shape[0]
    if i_end is None:
        i_end = N
    if counts is None:
        counts = np.zeros(nbins, np.int64)
    lib().orc_gr_counts(int(N), float(L), _dptr(x), _dptr(y), float(sigma), float(dr),
                        int(nbins), int(i_begin), int(i_end),
                        counts.ctypes.data_as(C.POINTER(C.c_int64)))
    return counts


def gr_counts_cells(L, x, y, sigma, dr, nbins, counts=None):
    """gr_counts over all disks, pairs found through a cell list (same
    counts; for large N)."""
    N = x.shape[0]
    if counts is None:
        counts = np.zeros(nbins, np.int64)
    lib().orc_gr_counts_cells(int(N), float(L), _dptr(x), _dptr(y), float(sigma), float(dr),
                              int(nbins), counts.ctypes.data_as(C.POINTER(C.c_int64)))
    return counts


def hexatic(L, x, y, rs=3.5):
    """Hexatic order parameter (eq. Psi) with Delaunay next neighbours.
    Returns (Psi as a complex number, per-disk Psi_k as complex array,
    neighbour counts, number of disks whose Voronoi cell was not certified)."""
    N = x.shape[0]
    pk = np.empty(2 * N)
    nn = np.empty(N, np.int32)
    ps = np.empty(2)
    bad = lib().orc_hexatic(int(N), float(L), _dptr(x), _dptr(y), float(rs),
                            pk.ctypes.data, nn.ctypes.data, ps.ctypes.data)
    if bad < 0:
        raise ValueError("box too small for the neighbour radius")
    return complex(ps[0], ps[1]), pk[0::2] + 1j * pk[1::2], nn, bad


def min_dist2(L, x, y, rcut=2.0):
    return lib().orc_min_dist2(int(x.shape[0]), float(L), _dptr(x), _dptr(y), float(rcut))


def run_chain_frame(X, Y, n_mem, m, dx, dy, ell, w, h, sigma=1.0, ids=None, imgs=None,
                    specular=False, reject=False):
    """One chain on an explicit frame; returns (X, Y, stats, record)."""
    X = np.ascontiguousarray(X, dtype=np.float64).copy()
    Y = np.ascontiguousarray(Y, dtype=np.float64).copy()
    n = X.shape[0]
    ids = np.arange(n, dtype=np.int64) if ids is None else np.asarray(ids, np.int64)
    imgs = np.full(n, 4, np.int32) if imgs is None else np.asarray(imgs, np.int32)
    st = Stats()
    rec = np.zeros(1, CHAIN_REC)
    rc = lib().orc_run_chain_frame(n, int(n_mem), _dptr(X), _dptr(Y),
                                   ids.ctypes.data_as(C.POINTER(C.c_int64)),
                                   imgs.ctypes.data_as(C.POINTER(C.c_int32)), float(w), float(h),
                                   float(sigma), int(m), float(dx), float(dy), float(ell),
                                   int(bool(specular)) | 2 * int(bool(reject)), C.byref(st),
                                   rec.ctypes.data_as(C.c_void_p))
    if rc != 0:
        raise ValueError("bad frame")
    return X, Y, st, rec[0]


def gr_normalise(counts, n_meas, N, L, sigma, dr):
    """g(R_i) = <n(r_i)> / (N rho 2 pi R_i dr) with the area-weighted radius
    R_i of each bin (Sec. 2); bins span [sigma + i dr, sigma + (i+1) dr)."""
    nb = counts.shape[0]
    e0 = sigma + dr * np.arange(nb)
    e1 = e0 + dr
    R = 2.0 * (e1**3 - e0**3) / (3.0 * (e1**2 - e0**2))
    rho = N / (L * L)
    g = (counts / float(n_meas)) / (N * rho * 2.0 * math.pi * R * dr)
    return R, g


def pressure_from_sums(sum_b, sum_disp, N, L, sigma):
    """beta P sigma^2 = rho sigma^2 (1 + sum_b / sum_disp): collision form of
    eq. (pressure)."""
    rho = N / (L * L)
    return rho * sigma * sigma * (1.0 + sum_b / sum_disp)


def pressure_from_gcontact(g_contact, N, L, sigma):
    """eq. (pressure): beta P sigma^2 = sigma^2 rho (1 + pi/2 sigma^2 rho g(sigma+))."""
    rho = N / (L * L)
    return sigma * sigma * rho * (1.0 + 0.5 * math.pi * sigma * sigma * rho * g_contact)


# ---- striped decomposition (Fig. 3 "stripes") -----------------------------

def stripe_draws(p, t):
    """(shift across the axis, colour that runs first) of sweep t."""
    sh, first = C.c_double(), C.c_int()
    lib().orc_stripe_draws(C.byref(p), int(t), C.byref(sh), C.byref(first))
    return sh.value, first.value


def stripe_bin(p, t, x, y):
    out = np.empty(p.N, np.int32)
    rc = lib().orc_stripe_bin(C.byref(p), int(t), _dptr(x), _dptr(y),
                              out.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    return out


def stripe_sweeps(p, x, y, t0, n_sweeps, stats=None, records=False):
    """Sweeps of the striped decomposition in place on x, y (p.cells_x
    stripes).  Returns (stats, records [n_sweeps, stripes, n_m] or None)."""
    st = stats if stats is not None else Stats()
    recs = None
    rp = None
    if records:
        recs = np.zeros((n_sweeps, p.cells_x, p.n_m), CHAIN_REC)
        rp = recs.ctypes.data_as(C.c_void_p)
    rc = lib().orc_stripe_sweeps(C.byref(p), _dptr(x), _dptr(y), int(t0), int(n_sweeps),
                                 C.byref(st), rp)
    if rc != 0:
        raise ValueError("oracle rejected the parameters (rc=%d)" % rc)
    return st, recs


def run_chain_stripe(U, V, n_mem, m, sign, ell, L, sigma=1.0, keys=None, reject=True):
    """One chain on an explicit stripe frame; returns (U, stats, record, rejected)."""
    U = np.ascontiguousarray(U, dtype=np.float64).copy()
    V = np.ascontiguousarray(V, dtype=np.float64).copy()
    n = U.shape[0]
    keys = np.arange(n, dtype=np.int64) if keys is None else np.asarray(keys, np.int64)
    st = Stats()
    rec = np.zeros(1, CHAIN_REC)
    rc = lib().orc_run_chain_stripe(n, int(n_mem), _dptr(U), _dptr(V),
                                    keys.ctypes.data_as(C.POINTER(C.c_int64)), float(L),
                                    float(sigma), int(m), int(sign), float(ell), int(reject),
                                    C.byref(st), rec.ctypes.data_as(C.c_void_p))
    if rc < 0:
        raise ValueError("bad frame")
    return U, st, rec[0], rc == 1


# ---- three dimensions ------------------------------------------------------

def make_params3(N, L, sigma, cells, ell, n_m, seed, replica=0, flags=0):
    return Params3(int(N), float(L), float(sigma), int(cells), float(ell), int(n_m), int(seed),
                   int(replica), int(flags))


def sweep_draws3(p, t):
    sh = (C.c_double * 3)()
    perm = (C.c_int * 8)()
    lib().orc3_sweep_draws(C.byref(p), int(t), sh, perm)
    return list(sh), list(perm)


def bin_cells3(p, t, x, y, z):
    cell = np.empty(p.N, np.int32)
    rc = lib().orc3_bin(C.byref(p), int(t), _dptr(x), _dptr(y), _dptr(z),
                        cell.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    return cell


def sweeps3(p, x, y, z, t0, n_sweeps, stats=None, records=False):
    """Three-dimensional sweeps in place on x, y, z (float64, id order).
    Returns (stats, records [n_sweeps, cells^3, n_m] or None)."""
    st = stats if stats is not None else Stats()
    recs = None
    rp = None
    if records:
        recs = np.zeros((n_sweeps, p.cells ** 3, p.n_m), CHAIN_REC)
        rp = recs.ctypes.data_as(C.c_void_p)
    rc = lib().orc3_sweeps(C.byref(p), _dptr(x), _dptr(y), _dptr(z), int(t0), int(n_sweeps),
                           C.byref(st), rp)
    if rc != 0:
        raise ValueError("oracle rejected the parameters (rc=%d)" % rc)
    return st, recs


def run_chain_frame3(X, Y, Z, n_mem, m, axis, sign, ell, w, sigma=1.0, ids=None, imgs=None):
    """One three-dimensional chain on an explicit frame; returns
    (X, Y, Z, stats, record)."""
    X = np.ascontiguousarray(X, dtype=np.float64).copy()
    Y = np.ascontiguousarray(Y, dtype=np.float64).copy()
    Z = np.ascontiguousarray(Z, dtype=np.float64).copy()
    n = X.shape[0]
    ids = np.arange(n, dtype=np.int64) if ids is None else np.asarray(ids, np.int64)
    imgs = np.full(n, 13, np.int32) if imgs is None else np.asarray(imgs, np.int32)
    st = Stats()
    rec = np.zeros(1, CHAIN_REC)
    rc = lib().orc3_run_chain_frame(n, int(n_mem), _dptr(X), _dptr(Y), _dptr(Z),
                                    ids.ctypes.data_as(C.POINTER(C.c_int64)),
                                    imgs.ctypes.data_as(C.POINTER(C.c_int32)), float(w),
                                    float(sigma), int(m), int(axis), int(sign), float(ell),
                                    C.byref(st), rec.ctypes.data_as(C.c_void_p))
    if rc != 0:
        raise ValueError("bad frame")
    return X, Y, Z, st, rec[0]


def min_dist2_3(L, x, y, z, rcut=2.0):
    return lib().orc3_min_dist2(int(x.shape[0]), float(L), _dptr(x), _dptr(y), _dptr(z),
                                float(rcut))


def pressure_from_sums3(sum_b_w, sum_disp_w, N, L, sigma):
    """beta P sigma^3 = rho sigma^3 (1 + sum_b_w / sum_disp_w)."""
    rho = N / L**3
    return rho * sigma**3 * (1.0 + sum_b_w / sum_disp_w)
