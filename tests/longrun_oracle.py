"""Oracle side of the long-run statistical comparison (tests/test_gpu_longrun.py).

One independent oracle run per call: square-lattice start, `melt` untimed
sweeps, then `sweeps` measured sweeps with the member-weighted collision
pressure accumulated over them and the ordered-pair histogram taken every
`gr_every` sweeps.  Kept apart from the test module so that worker processes
started with `spawn` import only numpy and the oracle (no torch, no CUDA).
"""
import time

import numpy as np

import ecmc_workloads as W
import oracle


def run(N, eta, cells, ell, n_m, seed, replica, melt, sweeps, gr_every, dr, nbins):
    t_start = time.time()
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, cells, cells, ell, n_m, seed, replica)
    oracle.sweeps(p, x, y, 0, melt)
    st = oracle.Stats()
    counts = np.zeros(nbins, np.int64)
    n_meas = 0
    t = melt
    while t < melt + sweeps:
        k = min(gr_every, melt + sweeps - t)
        oracle.sweeps(p, x, y, t, k, stats=st)
        t += k
        if k == gr_every:
            oracle.gr_counts_cells(L, x, y, 1.0, dr, nbins, counts=counts)
            n_meas += 1
    rho = N / (L * L)
    return {"P": rho * (1.0 + st.sum_b_w / st.sum_disp_w), "counts": counts, "n_meas": n_meas,
            "events": int(st.events), "seconds": time.time() - t_start, "x": x, "y": y}
