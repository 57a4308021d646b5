"""Parity of the rejecting boundary rule (ECMC_BOUNDARY_REJECT; the
comparison variant of Sec. 3.4 and Fig. 3) with the oracle's
ORC_BOUNDARY_REJECT, through the C ABI: positions to 1e-12 (bitwise in
practice), chain records, event counters and the count of rejected chains
exactly, on the persistent and the per-phase kernels, with FP32 screening and
all-FP64 candidates, with and without replacement.  From the square-lattice
start a chain longer than the lattice gap runs down a whole row into the wall,
so the budgets are short enough that some chains are accepted.  A budget longer than the
cell diagonal rejects every chain and must leave every coordinate as it was.
"""
import math

import numpy as np
import pytest

import ecmc_workloads as W
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1409_6948_gb300 import ecmc as E  # noqa: E402
from test_gpu_parity import make, run_pair  # noqa: E402

REJ = E.BOUNDARY_REJECT


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("N,eta,cells,ell,nm,sweeps", [
    (256, 0.70, 2, 0.3, 4, 10),
    (4096, 0.70, 8, 0.1, 8, 6),
    (4096, 0.50, 16, 1.0, 3, 6),
])
def test_rejection_matches_oracle(N, eta, cells, ell, nm, sweeps, prec, persistent):
    st = run_pair(N, eta, cells, cells, ell, nm, 11, sweeps, prec=prec,
                  persistent=persistent, boundary=REJ)
    assert 0 < st.rejected < st.chains


def test_rejection_with_shuffled_lists_matches_oracle():
    st = run_pair(4096, 0.70, 8, 8, 0.1, 6, 12, 5, list_mode=1, boundary=REJ)
    assert 0 < st.rejected < st.chains


def test_rejection_at_the_papers_fig3_size():
    # N = 256^2, eta = 0.708 with 32 x 32 cells (the setup of Fig. 3)
    st = run_pair(65536, 0.708, 32, 32, 0.1, 4, 13, 3, records=False, boundary=REJ)
    assert 0 < st.rejected < st.chains


def test_budget_beyond_the_cell_leaves_the_configuration_unchanged():
    N, eta, cells = 4096, 0.70, 8
    g, p, L = make(N, eta, cells, cells, 2.0, 4, 14)
    g.sweep(10)
    xy0 = g.positions().copy()
    g.close()
    ell = 1.5 * math.sqrt(2.0) * L / cells
    g, p, L = make(N, eta, cells, cells, ell, 4, 14, boundary=REJ)
    g.set_positions(xy0, t0=10)
    g.reset_stats()
    g.sweep(4)
    c = g.counters()
    assert c.rejected_chains == c.chains == 4 * cells * cells * 4
    assert c.sum_b == 0.0 and c.sum_disp == 0.0
    assert np.array_equal(g.positions(), xy0)
    g.close()


def test_rejection_needs_axis_chains():
    g, p, L = make(256, 0.70, 2, 2, 1.0, 2, 1, dir_mode=E.DIR_ISOTROPIC)
    with pytest.raises(E.EcmcError) as ei:
        g.set_param(E.PARAM_BOUNDARY, REJ)
    assert ei.value.code == E.ERR_UNSUPPORTED
    g.set_param(E.PARAM_DIR_MODE, 0)
    g.set_param(E.PARAM_BOUNDARY, REJ)
    with pytest.raises(E.EcmcError):
        g.set_param(E.PARAM_DIR_MODE, E.DIR_ISOTROPIC)
    g.close()
