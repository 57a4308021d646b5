"""Thin ctypes binding of libecmc.so (include/ecmc.h).

Argument marshalling only: every step of the sweep runs in the CUDA library.
The binding raises if the library cannot be loaded; there is no fallback.
Device buffers may be passed as torch CUDA tensors (their data pointer is
used); host buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_OVERLAP, ERR_TIMEOUT, ERR_STATE, ERR_CAPACITY, \
    ERR_UNSUPPORTED, ERR_CHAIN_CAP = -1, -2, -3, -4, -5, -6, -7, -8, -9

PARAM_N_CHAINS = 1
PARAM_DIR_MODE = 2
PARAM_PRECISION = 3
PARAM_REPLICA = 4
PARAM_LANES_PER_CELL = 5
PARAM_GR_DR = 6
PARAM_GR_RMAX = 7
PARAM_TIMING = 8
PARAM_STRIP_WIDTH = 9
PARAM_RECORD_CHAINS = 10
PARAM_WARPS_PER_BLOCK = 11
PARAM_USE_GRAPH = 12
PARAM_FRAME_MODE = 13
PARAM_REPLAY = 14
PARAM_PERSISTENT = 15
PARAM_WAIT_LIMIT_MS = 16
PARAM_WAIT_TEST = 17
PARAM_KERNELS_PER_SWEEP = 18
PARAM_LIST_MODE = 19
PARAM_CHAINS_IN_FLIGHT = 20
PARAM_BOUNDARY = 21
BOUNDARY_REFLECT = 0
BOUNDARY_REJECT = 1
LIST_WITH_REPL = 0
LIST_WITHOUT_REPL = 1

DIR_PM_AXIS_ALT = 0
DIR_POS_ONLY = 1
DIR_ISOTROPIC = 2
PREC_FP64 = 0
PREC_FP32_GEOM = 1
TUNE_EVENTS = 0
TUNE_MSD = 1
TUNE_TAU = 2


class Counters(C.Structure):
    _fields_ = [("sweeps", C.c_int64), ("chains", C.c_int64), ("events", C.c_int64),
                ("lifts", C.c_int64), ("frozen_hits", C.c_int64), ("wall_hits", C.c_int64),
                ("fp64_evals", C.c_int64), ("sum_b", C.c_double), ("sum_disp", C.c_double),
                ("replayed_legs", C.c_int64), ("rejected_chains", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Timing(C.Structure):
    _fields_ = [("bin_ms", C.c_double), ("frame_ms", C.c_double), ("phase_ms", C.c_double),
                ("other_ms", C.c_double), ("bin_launches", C.c_int64),
                ("frame_launches", C.c_int64), ("phase_launches", C.c_int64),
                ("other_launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneResult(C.Structure):
    _fields_ = [("lanes_per_cell", C.c_int), ("warps_per_block", C.c_int),
                ("frame_mode", C.c_int), ("persistent", C.c_int),
                ("ms_per_sweep", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GeomTrial(C.Structure):
    _fields_ = [("cells", C.c_int), ("n_m", C.c_int), ("ell", C.c_double), ("status", C.c_int),
                ("sweeps", C.c_int64), ("ms_per_sweep", C.c_double),
                ("events_per_s", C.c_double), ("sweeps_per_s", C.c_double),
                ("lambda0", C.c_double), ("ell_star", C.c_double),
                ("msd_per_sweep", C.c_double), ("tau_sweeps", C.c_double),
                ("score", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ReplicaDesc(C.Structure):
    _fields_ = [("N", C.c_int64), ("L", C.c_double), ("sigma", C.c_double),
                ("cells_x", C.c_int), ("cells_y", C.c_int), ("ell", C.c_double),
                ("n_m", C.c_int), ("seed", C.c_uint64), ("replica", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


CHAIN_REC = np.dtype([("start_id", np.int64), ("end_id", np.int64), ("events", np.int64),
                      ("walls", np.int64)])

# every symbol the header declares, with (restype, argtypes)
_H = C.c_void_p
_SIGS = {
    "ecmc_create": (C.c_int, [C.POINTER(_H), C.c_int64, C.c_double, C.c_double, C.c_int, C.c_int,
                              C.c_double, C.c_uint64]),
    "ecmc_create_batch": (C.c_int, [C.POINTER(_H), C.POINTER(ReplicaDesc), C.c_int]),
    "ecmc_num_replicas": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "ecmc_replica_desc": (C.c_int, [_H, C.c_int, C.POINTER(ReplicaDesc)]),
    "ecmc_replica_pressure": (C.c_int, [_H, C.c_int, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]),
    "ecmc_replica_counters": (C.c_int, [_H, C.c_int, C.POINTER(Counters)]),
    "ecmc_suggest_parameters": (C.c_int, [C.c_int64, C.c_double, C.c_double, C.c_double,
                                          C.POINTER(ReplicaDesc)]),
    "ecmc_tune_geometry": (C.c_int, [C.POINTER(ReplicaDesc), C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                     C.POINTER(GeomTrial), C.POINTER(C.c_int)]),
    "ecmc_autotune": (C.c_int, [_H, C.c_int, C.POINTER(TuneResult), C.POINTER(TuneResult),
                                C.c_int, C.POINTER(C.c_int)]),
    "ecmc_destroy": (C.c_int, [_H]),
    "ecmc_set_param": (C.c_int, [_H, C.c_int, C.c_double]),
    "ecmc_get_param": (C.c_int, [_H, C.c_int, C.POINTER(C.c_double)]),
    "ecmc_set_stream": (C.c_int, [_H, C.c_void_p]),
    "ecmc_set_positions": (C.c_int, [_H, C.c_void_p, C.c_int, C.c_int64]),
    "ecmc_sweep": (C.c_int, [_H, C.c_int64]),
    "ecmc_synchronize": (C.c_int, [_H]),
    "ecmc_positions": (C.c_int, [_H, C.c_void_p, C.c_int]),
    "ecmc_sweep_index": (C.c_int, [_H, C.POINTER(C.c_int64)]),
    "ecmc_counters": (C.c_int, [_H, C.POINTER(Counters)]),
    "ecmc_reset_stats": (C.c_int, [_H]),
    "ecmc_pressure": (C.c_int, [_H, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ecmc_gr_measure": (C.c_int, [_H]),
    "ecmc_gr_counts": (C.c_int, [_H, C.c_void_p, C.c_int, C.POINTER(C.c_int64)]),
    "ecmc_gr": (C.c_int, [_H, C.c_void_p, C.c_void_p, C.c_int]),
    "ecmc_gr_nbins": (C.c_int, [_H, C.POINTER(C.c_int)]),
    "ecmc_replica_gr_measure": (C.c_int, [_H, C.c_int]),
    "ecmc_replica_gr_counts": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_int,
                                         C.POINTER(C.c_int64)]),
    "ecmc_replica_gr": (C.c_int, [_H, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "ecmc_min_distance": (C.c_int, [_H, C.POINTER(C.c_double)]),
    "ecmc_last_cells": (C.c_int, [_H, C.c_void_p]),
    "ecmc_kernel_times": (C.c_int, [_H, C.POINTER(Timing)]),
    "ecmc_chain_records": (C.c_int, [_H, C.c_void_p, C.c_int64]),
    "ecmc_device_peaks": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ecmc_sqrt_rn": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_double,
                               C.c_void_p]),
    "ecmc_hexatic": (C.c_int, [_H, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(C.c_int64)]),
    "ecmc_autocorrelation_time": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_int64,
                                            C.POINTER(C.c_double), C.c_void_p]),
    "ecmc_sweep_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_int,
                                     C.c_int, C.c_double, C.c_int, C.c_uint64, C.c_uint64,
                                     C.c_int64, C.c_int64, C.c_void_p]),
    "ecmc3_create": (C.c_int, [C.POINTER(_H), C.c_int64, C.c_double, C.c_double, C.c_int,
                               C.c_double, C.c_uint64]),
    "ecmc3_destroy": (C.c_int, [_H]),
    "ecmc3_set_param": (C.c_int, [_H, C.c_int, C.c_double]),
    "ecmc3_get_param": (C.c_int, [_H, C.c_int, C.POINTER(C.c_double)]),
    "ecmc3_set_stream": (C.c_int, [_H, C.c_void_p]),
    "ecmc3_set_positions": (C.c_int, [_H, C.c_void_p, C.c_int, C.c_int64]),
    "ecmc3_positions": (C.c_int, [_H, C.c_void_p, C.c_int]),
    "ecmc3_sweep": (C.c_int, [_H, C.c_int64]),
    "ecmc3_synchronize": (C.c_int, [_H]),
    "ecmc3_sweep_index": (C.c_int, [_H, C.POINTER(C.c_int64)]),
    "ecmc3_counters": (C.c_int, [_H, C.POINTER(Counters)]),
    "ecmc3_pressure": (C.c_int, [_H, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ecmc3_reset_stats": (C.c_int, [_H]),
    "ecmc3_min_distance": (C.c_int, [_H, C.POINTER(C.c_double)]),
    "ecmc3_last_cells": (C.c_int, [_H, C.c_void_p]),
    "ecmc3_chain_records": (C.c_int, [_H, C.c_void_p]),
    "ecmc_stripes_create": (C.c_int, [C.POINTER(_H), C.c_int64, C.c_double, C.c_double, C.c_int,
                                      C.c_double, C.c_uint64]),
    "ecmc_stripes_destroy": (C.c_int, [_H]),
    "ecmc_stripes_set_param": (C.c_int, [_H, C.c_int, C.c_double]),
    "ecmc_stripes_get_param": (C.c_int, [_H, C.c_int, C.POINTER(C.c_double)]),
    "ecmc_stripes_set_stream": (C.c_int, [_H, C.c_void_p]),
    "ecmc_stripes_set_positions": (C.c_int, [_H, C.c_void_p, C.c_int, C.c_int64]),
    "ecmc_stripes_positions": (C.c_int, [_H, C.c_void_p, C.c_int]),
    "ecmc_stripes_sweep": (C.c_int, [_H, C.c_int64]),
    "ecmc_stripes_synchronize": (C.c_int, [_H]),
    "ecmc_stripes_sweep_index": (C.c_int, [_H, C.POINTER(C.c_int64)]),
    "ecmc_stripes_counters": (C.c_int, [_H, C.POINTER(Counters)]),
    "ecmc_stripes_pressure": (C.c_int, [_H, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ecmc_stripes_reset_stats": (C.c_int, [_H]),
    "ecmc_stripes_last_stripes": (C.c_int, [_H, C.c_void_p]),
    "ecmc_stripes_chain_records": (C.c_int, [_H, C.c_void_p]),
    "ecmc_strerror": (C.c_char_p, [C.c_int]),
    "ecmc_last_error_message": (C.c_char_p, []),
    "ecmc_version": (C.c_char_p, []),
}

_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libecmc.so (building it first if needed and allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libecmc.so is not built (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class EcmcError(RuntimeError):
    def __init__(self, code, where):
        lib = load()
        msg = lib.ecmc_strerror(code).decode()
        detail = lib.ecmc_last_error_message().decode()
        super().__init__("%s: %s (%d): %s" % (where, msg, code, detail))
        self.code = code


def _check(rc, where):
    if rc != OK:
        raise EcmcError(rc, where)


def _ptr(buf):
    """(address, on_device) of a numpy array or torch tensor."""
    if hasattr(buf, "data_ptr"):
        return C.c_void_p(buf.data_ptr()), 1 if buf.is_cuda else 0
    assert buf.flags.c_contiguous
    return C.c_void_p(buf.ctypes.data), 0


class Ecmc:
    """One hard-disk system on the GPU (a handle of the C library)."""

    def __init__(self, N, L, sigma, cells_x, cells_y, ell, seed):
        lib = load()
        h = _H()
        _check(lib.ecmc_create(C.byref(h), int(N), float(L), float(sigma), int(cells_x),
                               int(cells_y), float(ell), C.c_uint64(int(seed))), "ecmc_create")
        self._h = h
        self.N, self.L, self.sigma = int(N), float(L), float(sigma)
        self.cells_x, self.cells_y = int(cells_x), int(cells_y)
        self.R = 1

    @classmethod
    def batch(cls, descs):
        """A handle with several independent replicas; descs are dicts with the
        fields of ecmc_replica_desc_t (n_m = 0 picks eq. nm)."""
        lib = load()
        arr = (ReplicaDesc * len(descs))()
        for i, d in enumerate(descs):
            arr[i] = ReplicaDesc(int(d["N"]), float(d["L"]), float(d.get("sigma", 1.0)),
                                 int(d["cells_x"]), int(d.get("cells_y", d["cells_x"])),
                                 float(d["ell"]), int(d.get("n_m", 0)), int(d["seed"]),
                                 int(d.get("replica", 0)))
        h = _H()
        _check(lib.ecmc_create_batch(C.byref(h), arr, len(descs)), "ecmc_create_batch")
        self = cls.__new__(cls)
        self._h = h
        self.R = len(descs)
        self.N = sum(int(d["N"]) for d in descs)
        self.L, self.sigma = float(descs[0]["L"]), float(descs[0].get("sigma", 1.0))
        self.cells_x = int(descs[0]["cells_x"])
        self.cells_y = int(descs[0].get("cells_y", descs[0]["cells_x"]))
        return self

    def autotune(self, trial_sweeps=3):
        """Measure every launch shape, keep the fastest (state unchanged)."""
        best = TuneResult()
        arr = (TuneResult * 64)()
        n = C.c_int()
        _check(load().ecmc_autotune(self._h, int(trial_sweeps), C.byref(best), arr, 64,
                                    C.byref(n)), "ecmc_autotune")
        return best.as_dict(), [arr[i].as_dict() for i in range(n.value)]

    def hexatic(self, rs=0.0, per_disk=False):
        """Hexatic order parameter (eq. Psi) with Delaunay next neighbours.
        Returns Psi (complex; an array of one per replica for a batch), or
        (Psi, Psi_k complex array, neighbour counts, uncertified disks) with
        per_disk."""
        R = self.num_replicas()
        N = sum(self.replica_desc(r)["N"] for r in range(R))
        psi = np.empty(2 * R)
        nbad = C.c_int64()
        pk = np.empty(2 * N) if per_disk else None
        nn = np.empty(N, np.int32) if per_disk else None
        _check(load().ecmc_hexatic(self._h, float(rs), psi.ctypes.data,
                                   pk.ctypes.data if per_disk else None,
                                   nn.ctypes.data if per_disk else None, C.byref(nbad)),
               "ecmc_hexatic")
        z = psi[0::2] + 1j * psi[1::2]
        z = complex(z[0]) if R == 1 else z
        if not per_disk:
            return z
        return z, pk[0::2] + 1j * pk[1::2], nn, nbad.value

    def replica_desc(self, r):
        d = ReplicaDesc()
        _check(load().ecmc_replica_desc(self._h, int(r), C.byref(d)), "ecmc_replica_desc")
        return d.as_dict()

    def num_replicas(self):
        n = C.c_int()
        _check(load().ecmc_num_replicas(self._h, C.byref(n)), "ecmc_num_replicas")
        return n.value

    def replica_pressure(self, r):
        p, se = C.c_double(), C.c_double()
        _check(load().ecmc_replica_pressure(self._h, int(r), C.byref(p), C.byref(se)),
               "ecmc_replica_pressure")
        return p.value, se.value

    def replica_counters(self, r):
        c = Counters()
        _check(load().ecmc_replica_counters(self._h, int(r), C.byref(c)), "ecmc_replica_counters")
        return c

    def close(self):
        if getattr(self, "_h", None):
            load().ecmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # parameters
    def set_param(self, key, value):
        _check(load().ecmc_set_param(self._h, int(key), float(value)), "ecmc_set_param")

    def get_param(self, key):
        v = C.c_double()
        _check(load().ecmc_get_param(self._h, int(key), C.byref(v)), "ecmc_get_param")
        return v.value

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an integer cudaStream_t, or None."""
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        _check(load().ecmc_set_stream(self._h, C.c_void_p(stream or 0)), "ecmc_set_stream")

    # configuration
    def set_positions(self, xy, t0=0):
        p, dev = _ptr(xy)
        _check(load().ecmc_set_positions(self._h, p, dev, int(t0)), "ecmc_set_positions")

    def positions(self, out=None):
        if out is None:
            out = np.empty(2 * self.N, np.float64)
        p, dev = _ptr(out)
        _check(load().ecmc_positions(self._h, p, dev), "ecmc_positions")
        return out

    def sweep(self, n=1):
        _check(load().ecmc_sweep(self._h, int(n)), "ecmc_sweep")

    def synchronize(self):
        _check(load().ecmc_synchronize(self._h), "ecmc_synchronize")

    def sweep_index(self):
        t = C.c_int64()
        _check(load().ecmc_sweep_index(self._h, C.byref(t)), "ecmc_sweep_index")
        return t.value

    # measurements
    def counters(self):
        c = Counters()
        _check(load().ecmc_counters(self._h, C.byref(c)), "ecmc_counters")
        return c

    def reset_stats(self):
        _check(load().ecmc_reset_stats(self._h), "ecmc_reset_stats")

    def pressure(self):
        p, se = C.c_double(), C.c_double()
        _check(load().ecmc_pressure(self._h, C.byref(p), C.byref(se)), "ecmc_pressure")
        return p.value, se.value

    def gr_measure(self, replica=None):
        """Add the current configuration to the pair histogram of replica 0
        (default), of one replica, or of every replica (replica=-1)."""
        if replica is None:
            _check(load().ecmc_gr_measure(self._h), "ecmc_gr_measure")
        else:
            _check(load().ecmc_replica_gr_measure(self._h, int(replica)),
                   "ecmc_replica_gr_measure")

    def gr_nbins(self):
        n = C.c_int()
        _check(load().ecmc_gr_nbins(self._h, C.byref(n)), "ecmc_gr_nbins")
        return n.value

    def gr_counts(self, replica=0):
        nb = self.gr_nbins()
        out = np.zeros(nb, np.int64)
        nm = C.c_int64()
        _check(load().ecmc_replica_gr_counts(self._h, int(replica), C.c_void_p(out.ctypes.data),
                                             nb, C.byref(nm)), "ecmc_replica_gr_counts")
        return out, nm.value

    def gr(self, replica=0):
        nb = self.gr_nbins()
        g = np.zeros(nb)
        r = np.zeros(nb)
        _check(load().ecmc_replica_gr(self._h, int(replica), C.c_void_p(g.ctypes.data),
                                      C.c_void_p(r.ctypes.data), nb), "ecmc_replica_gr")
        return r, g

    def min_distance(self):
        d = C.c_double()
        _check(load().ecmc_min_distance(self._h, C.byref(d)), "ecmc_min_distance")
        return d.value

    def last_cells(self):
        out = np.empty(self.N, np.int32)
        _check(load().ecmc_last_cells(self._h, C.c_void_p(out.ctypes.data)), "ecmc_last_cells")
        return out

    def kernel_times(self):
        t = Timing()
        _check(load().ecmc_kernel_times(self._h, C.byref(t)), "ecmc_kernel_times")
        return t

    def chain_records(self):
        nm = int(self.get_param(PARAM_N_CHAINS))
        n = self.cells_x * self.cells_y * nm
        out = np.zeros(n, CHAIN_REC)
        _check(load().ecmc_chain_records(self._h, C.c_void_p(out.ctypes.data), n),
               "ecmc_chain_records")
        return out.reshape(self.cells_x * self.cells_y, nm)


PARAM3_N_CHAINS = 1
PARAM3_REPLICA = 4
PARAM3_PERSISTENT = 15
PARAM3_WAIT_LIMIT_MS = 16
PARAM3_WAIT_TEST = 17
PARAM3_REPLAY = 14


class Ecmc3:
    """One hard-sphere system on the GPU (three dimensions; include/ecmc3.h):
    N = k^3 spheres of diameter sigma in a periodic cube of side L, cells^3
    cubic cells, chains of displacement ell, simple cubic lattice start."""

    def __init__(self, N, L, sigma, cells, ell, seed):
        lib = load()
        h = _H()
        _check(lib.ecmc3_create(C.byref(h), int(N), float(L), float(sigma), int(cells),
                                float(ell), C.c_uint64(int(seed))), "ecmc3_create")
        self._h = h
        self.N, self.L, self.sigma, self.cells = int(N), float(L), float(sigma), int(cells)

    def close(self):
        if getattr(self, "_h", None):
            load().ecmc3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_param(self, key, value):
        _check(load().ecmc3_set_param(self._h, int(key), float(value)), "ecmc3_set_param")

    def get_param(self, key):
        v = C.c_double()
        _check(load().ecmc3_get_param(self._h, int(key), C.byref(v)), "ecmc3_get_param")
        return v.value

    def set_stream(self, stream):
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        _check(load().ecmc3_set_stream(self._h, C.c_void_p(stream or 0)), "ecmc3_set_stream")

    def set_positions(self, xyz, t0=0):
        p, dev = _ptr(xyz)
        _check(load().ecmc3_set_positions(self._h, p, dev, int(t0)), "ecmc3_set_positions")

    def positions(self, out=None):
        if out is None:
            out = np.empty(3 * self.N)
        p, dev = _ptr(out)
        _check(load().ecmc3_positions(self._h, p, dev), "ecmc3_positions")
        return out

    def sweep(self, n=1):
        _check(load().ecmc3_sweep(self._h, int(n)), "ecmc3_sweep")

    def synchronize(self):
        _check(load().ecmc3_synchronize(self._h), "ecmc3_synchronize")

    def sweep_index(self):
        t = C.c_int64()
        _check(load().ecmc3_sweep_index(self._h, C.byref(t)), "ecmc3_sweep_index")
        return t.value

    def counters(self):
        c = Counters()
        _check(load().ecmc3_counters(self._h, C.byref(c)), "ecmc3_counters")
        return c

    def pressure(self):
        p, se = C.c_double(), C.c_double()
        _check(load().ecmc3_pressure(self._h, C.byref(p), C.byref(se)), "ecmc3_pressure")
        return p.value, se.value

    def reset_stats(self):
        _check(load().ecmc3_reset_stats(self._h), "ecmc3_reset_stats")

    def min_distance(self):
        d = C.c_double()
        _check(load().ecmc3_min_distance(self._h, C.byref(d)), "ecmc3_min_distance")
        return d.value

    def last_cells(self):
        out = np.empty(self.N, np.int32)
        _check(load().ecmc3_last_cells(self._h, C.c_void_p(out.ctypes.data)),
               "ecmc3_last_cells")
        return out

    def chain_records(self):
        """Records of the last sweep: [cells^3, n_m] of (start_id, end_id,
        events, walls)."""
        nm = int(self.get_param(PARAM3_N_CHAINS))
        out = np.empty((self.cells ** 3, nm, 4), np.int32)
        _check(load().ecmc3_chain_records(self._h, C.c_void_p(out.ctypes.data)),
               "ecmc3_chain_records")
        return out


PARAM_STRIPES_N_CHAINS = 1
PARAM_STRIPES_REPLICA = 4
PARAM_STRIPES_BOUNDARY = 21
PARAM_STRIPES_LIST_MODE = 19
PARAM_STRIPES_KERNEL = 24


class EcmcStripes:
    """One hard-disk system swept with the striped decomposition of Fig. 3
    (include/ecmc_stripes.h): N = k^2 disks in a periodic square of side L,
    `stripes` stripes parallel to the chain axis, chains of displacement
    ell, rejected at a frozen disk by default; square lattice start."""

    def __init__(self, N, L, sigma, stripes, ell, seed):
        lib = load()
        h = _H()
        _check(lib.ecmc_stripes_create(C.byref(h), int(N), float(L), float(sigma), int(stripes),
                                       float(ell), C.c_uint64(int(seed))), "ecmc_stripes_create")
        self._h = h
        self.N, self.L, self.sigma, self.stripes = int(N), float(L), float(sigma), int(stripes)

    def close(self):
        if getattr(self, "_h", None):
            load().ecmc_stripes_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_param(self, key, value):
        _check(load().ecmc_stripes_set_param(self._h, int(key), float(value)),
               "ecmc_stripes_set_param")

    def get_param(self, key):
        v = C.c_double()
        _check(load().ecmc_stripes_get_param(self._h, int(key), C.byref(v)),
               "ecmc_stripes_get_param")
        return v.value

    def set_stream(self, stream):
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        _check(load().ecmc_stripes_set_stream(self._h, C.c_void_p(stream or 0)),
               "ecmc_stripes_set_stream")

    def set_positions(self, xy, t0=0):
        p, dev = _ptr(xy)
        _check(load().ecmc_stripes_set_positions(self._h, p, dev, int(t0)),
               "ecmc_stripes_set_positions")

    def positions(self, out=None):
        if out is None:
            out = np.empty(2 * self.N)
        p, dev = _ptr(out)
        _check(load().ecmc_stripes_positions(self._h, p, dev), "ecmc_stripes_positions")
        return out

    def sweep(self, n=1):
        _check(load().ecmc_stripes_sweep(self._h, int(n)), "ecmc_stripes_sweep")

    def synchronize(self):
        _check(load().ecmc_stripes_synchronize(self._h), "ecmc_stripes_synchronize")

    def sweep_index(self):
        t = C.c_int64()
        _check(load().ecmc_stripes_sweep_index(self._h, C.byref(t)), "ecmc_stripes_sweep_index")
        return t.value

    def counters(self):
        c = Counters()
        _check(load().ecmc_stripes_counters(self._h, C.byref(c)), "ecmc_stripes_counters")
        return c

    def pressure(self):
        p, se = C.c_double(), C.c_double()
        _check(load().ecmc_stripes_pressure(self._h, C.byref(p), C.byref(se)),
               "ecmc_stripes_pressure")
        return p.value, se.value

    def reset_stats(self):
        _check(load().ecmc_stripes_reset_stats(self._h), "ecmc_stripes_reset_stats")

    def last_stripes(self):
        out = np.empty(self.N, np.int32)
        _check(load().ecmc_stripes_last_stripes(self._h, C.c_void_p(out.ctypes.data)),
               "ecmc_stripes_last_stripes")
        return out

    def chain_records(self):
        """Records of the last sweep: [stripes, n_m] of (start_id, end_id,
        contacts, 0)."""
        nm = int(self.get_param(PARAM_STRIPES_N_CHAINS))
        out = np.empty((self.stripes, nm, 4), np.int32)
        _check(load().ecmc_stripes_chain_records(self._h, C.c_void_p(out.ctypes.data)),
               "ecmc_stripes_chain_records")
        return out


def version():
    return load().ecmc_version().decode()


def sweep_noalloc(xy, N, L, sigma, cells_x, cells_y, ell, n_m, seed, replica, t0, n_sweeps,
                  stream=None):
    """ecmc_sweep_noalloc: sweeps of caller-held device positions `xy` (a
    contiguous torch CUDA float64 tensor of at least 2N values on the current
    device, overwritten) using only the library's static scratch array; no
    device allocation."""
    import torch
    if not isinstance(xy, torch.Tensor) or not xy.is_cuda:
        raise ValueError("xy must be a CUDA tensor")
    if xy.dtype != torch.float64 or not xy.is_contiguous():
        raise ValueError("xy must be a contiguous float64 tensor")
    if xy.numel() < 2 * int(N):
        raise ValueError("xy holds %d values, 2N = %d needed" % (xy.numel(), 2 * int(N)))
    if xy.device.index != torch.cuda.current_device():
        raise ValueError("xy lives on cuda:%d, the current device is cuda:%d"
                         % (xy.device.index, torch.cuda.current_device()))
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(load().ecmc_sweep_noalloc(C.c_void_p(xy.data_ptr()), int(N), float(L), float(sigma),
                                     int(cells_x), int(cells_y), float(ell), int(n_m),
                                     C.c_uint64(int(seed)), C.c_uint64(int(replica)), int(t0),
                                     int(n_sweeps), C.c_void_p(stream or 0)),
           "ecmc_sweep_noalloc")


def tune_geometry(N, L, cells, ells, sigma=1.0, seed=0, replica=0, xy=None, warm_sweeps=10,
                  trial_sweeps=10, min_seconds=0.0, proxy=None):
    """ecmc_tune_geometry: one timed trial per (cells, ell), n_m from eq. nm;
    returns (trials as dicts in the order cells-major, index of the best)."""
    proxy = TUNE_MSD if proxy is None else proxy
    d = ReplicaDesc(int(N), float(L), float(sigma), 0, 0, 0.0, 0, int(seed), int(replica))
    cl = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
    el = np.ascontiguousarray(np.asarray(ells, dtype=np.float64))
    out = (GeomTrial * (cl.size * el.size))()
    best = C.c_int()
    buf = None
    if xy is not None:
        buf = np.ascontiguousarray(np.asarray(xy, dtype=np.float64))
    _check(load().ecmc_tune_geometry(C.byref(d), C.c_void_p(buf.ctypes.data) if buf is not None
                                     else None, C.c_void_p(cl.ctypes.data), int(cl.size),
                                     C.c_void_p(el.ctypes.data), int(el.size), int(warm_sweeps),
                                     int(trial_sweeps), float(min_seconds), int(proxy), out,
                                     C.byref(best)), "ecmc_tune_geometry")
    return [t.as_dict() for t in out], best.value


def suggest_parameters(N, L, sigma=1.0, min_cell_side=0.0):
    """The paper's three-step choice of cells, ell and n_m (Sec. 4)."""
    d = ReplicaDesc()
    _check(load().ecmc_suggest_parameters(int(N), float(L), float(sigma), float(min_cell_side),
                                          C.byref(d)), "ecmc_suggest_parameters")
    return d.as_dict()


def device_peaks():
    """(shared-memory GB/s, FP64 GFLOP/s) measured on the current device."""
    a, b = C.c_double(), C.c_double()
    _check(load().ecmc_device_peaks(C.byref(a), C.byref(b)), "ecmc_device_peaks")
    return a.value, b.value


def sqrt_rn(x, rel_error=None, stream=None):
    """The chain kernel's correctly rounded square root on an array.

    A float64 numpy array is evaluated on the host with the reciprocal
    square-root estimate perturbed by `rel_error` (|rel_error| <= 2^-20); a
    CUDA float64 tensor is evaluated on its device exactly as the kernel does.
    Returns an array (or tensor) of the same shape.
    """
    if isinstance(x, np.ndarray):
        xa = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty_like(xa)
        _check(load().ecmc_sqrt_rn(xa.ctypes.data, out.ctypes.data, xa.size, 0,
                                   float(rel_error or 0.0), None), "ecmc_sqrt_rn")
        return out
    if rel_error is not None:
        raise ValueError("rel_error applies to the host evaluation only")
    if not (x.is_cuda and x.dtype.is_floating_point and x.element_size() == 8):
        raise TypeError("expected a float64 numpy array or CUDA tensor")
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    xc = x.contiguous()
    out = xc.new_empty(xc.shape)
    _check(load().ecmc_sqrt_rn(C.c_void_p(xc.data_ptr()), C.c_void_p(out.data_ptr()),
                               xc.numel(), 1, 0.0, C.c_void_p(stream or 0)), "ecmc_sqrt_rn")
    return out


def autocorrelation_time(psi_series, max_lag=None):
    """Autocorrelation time tau of complex order-parameter series (eq. tau),
    computed by ecmc_autocorrelation_time: psi_series is one series [n] or R
    series [n, R] (replicas, averaged as the definition's <...>).  Returns
    (tau, C[0..max_lag])."""
    z = np.asarray(psi_series, dtype=complex)
    if z.ndim == 1:
        z = z[:, None]
    n, R = z.shape
    if max_lag is None:
        max_lag = n // 4
    buf = np.ascontiguousarray(np.stack([z.real, z.imag], -1).ravel())
    c = np.empty(int(max_lag) + 1)
    tau = C.c_double()
    _check(load().ecmc_autocorrelation_time(C.c_void_p(buf.ctypes.data), int(n), int(R),
                                            int(max_lag), C.byref(tau), C.c_void_p(c.ctypes.data)),
           "ecmc_autocorrelation_time")
    return tau.value, c

