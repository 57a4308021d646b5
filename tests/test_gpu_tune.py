"""ecmc_tune_geometry: the degree of parallelisation chosen by measurement
(Sec. 4).  Every trial runs with n_m from eq. (nm) (recomputed here by the
oracle's own rule), reports the measured mean free path and the criterion's
ell* from it, and the best trial maximises the chosen proxy."""
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


@pytest.mark.parametrize("proxy", [E.TUNE_MSD, E.TUNE_EVENTS])
def test_trials_and_choice(proxy):
    N, eta = 4096, 0.70
    L = W.box_side(N, eta)
    cells, ells = [4, 8, 16, 32, 34], [0.5, 2.0]  # 34 cells: side 1.88 sigma, skipped
    trials, best = E.tune_geometry(N, L, cells, ells, seed=3, warm_sweeps=10, trial_sweeps=6,
                                   min_seconds=0.0, proxy=proxy)
    assert len(trials) == len(cells) * len(ells)
    ran = [t for t in trials if t["status"] == 0]
    assert len(ran) == 8
    for t in trials:
        if t["cells"] == 34:
            assert t["status"] == E.ERR_ARG and t["score"] == -1.0
            continue
        assert t["n_m"] == oracle.default_nm(N, L, 1.0, t["cells"], t["cells"], t["ell"])
        assert t["events_per_s"] > 0 and t["sweeps"] >= 6
        assert 0.005 < t["lambda0"] < 0.3
        n = t["cells"] ** 2 / 4.0
        assert t["ell_star"] == pytest.approx(L * t["lambda0"] / math.sqrt(n), rel=1e-12)
        if proxy == E.TUNE_MSD:
            assert t["msd_per_sweep"] > 0
            assert t["score"] == pytest.approx(t["msd_per_sweep"] * t["sweeps_per_s"])
        else:
            assert t["score"] == pytest.approx(t["events_per_s"])
    assert best == int(np.argmax([t["score"] for t in trials]))


def test_tau_proxy_and_start_configuration():
    # from a given (melted) configuration; the tau proxy follows eq. tau on the
    # Psi series of the trial
    N, eta = 1024, 0.60
    L = W.box_side(N, eta)
    x, y = W.square_lattice(N, L)
    p = oracle.make_params(N, L, 1.0, 4, 4, 2.0, 2, 5)
    oracle.sweeps(p, x, y, 0, 30)
    xy = np.stack([x, y], 1).ravel()
    trials, best = E.tune_geometry(N, L, [4, 8], [1.0, 3.0], seed=5, xy=xy, warm_sweeps=5,
                                   trial_sweeps=80, proxy=E.TUNE_TAU)
    for t in trials:
        assert t["status"] == 0
        assert t["tau_sweeps"] > 0
        if math.isfinite(t["tau_sweeps"]):
            assert t["score"] == pytest.approx(t["sweeps_per_s"] / t["tau_sweeps"])
        else:
            assert t["score"] == 0.0
    assert best == int(np.argmax([t["score"] for t in trials]))


def test_bad_arguments():
    with pytest.raises(E.EcmcError):
        E.tune_geometry(256, 16.9, [2], [1.0], proxy=7)
    with pytest.raises(E.EcmcError):  # no candidate can run: cell side below 2 sigma
        E.tune_geometry(256, 16.9, [10], [1.0])
