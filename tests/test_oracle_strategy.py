"""Pins of the oracle's parameter strategy (the closing strategy of Sec. 4):
the largest square grid of 2x2 blocks with N / (eta n) > 100, ell from eq.
(criterion), n_m from eq. (nm); and the same choice as the CUDA library's
host-side ecmc_suggest_parameters, so that both benchmark arms run the same
workload."""
import math

import pytest

import ecmc_workloads as W
import oracle

TABLE = [(1048576, 0.72), (262144, 0.70), (4096, 0.60), (65536, 0.708), (4194304, 0.716),
         (4096, 0.704), (256, 0.70), (64, 0.70), (16384, 0.74), (100 * 100, 0.65)]


@pytest.mark.parametrize("N,eta", TABLE)
def test_three_steps(N, eta):
    L = W.box_side(N, eta)
    cells, ell, nm = oracle.suggest_parameters(N, L, 1.0, 2.0)
    h = cells // 2
    n = h * h
    eta_hcp = math.pi / (2 * math.sqrt(3))
    lam0 = (eta_hcp - eta) / (2 * eta_hcp)
    # step 1: n is the largest square number of blocks with N/(eta n) > 100,
    # unless the cell side (above 2 sigma here) forces fewer
    if N / (eta * n) > 100:
        assert N / (eta * (h + 1) ** 2) <= 100 or L / (2 * (h + 1)) <= 2.0
        assert ell > 10 * lam0 * 0.999999
    else:
        assert h == 1
    assert L / cells > 2.0
    # step 2: eq. (criterion)
    assert ell == pytest.approx(lam0 * math.sqrt(N / (eta * n)), rel=1e-12)
    # step 3: eq. (nm)
    assert nm == max(1, math.floor(N / (4 * n) * lam0 / ell + 0.5))


def test_paper_system_of_figs_5_and_6():
    # N = 64^2 at eta = 0.704: the strategy's n keeps ell above 10 lambda0
    N, eta = 4096, 0.704
    L = W.box_side(N, eta)
    cells, ell, nm = oracle.suggest_parameters(N, L)
    eta_hcp = math.pi / (2 * math.sqrt(3))
    lam0 = (eta_hcp - eta) / (2 * eta_hcp)
    assert cells == 14 and ell > 10 * lam0 and nm >= 1


def test_no_grid_fits():
    with pytest.raises(ValueError):
        oracle.suggest_parameters(16, W.box_side(16, 0.7), 1.0, 3.0)


@pytest.mark.parametrize("N,eta", TABLE)
def test_same_choice_as_the_library(N, eta):
    P = pytest.importorskip("paper_1409_6948_gb300")
    from paper_1409_6948_gb300 import ecmc as E
    try:
        P.load()
    except Exception as e:  # noqa: BLE001
        pytest.skip("library not built: %s" % e)
    L = W.box_side(N, eta)
    lib = E.suggest_parameters(N, L, 1.0, 2.0)
    cells, ell, nm = oracle.suggest_parameters(N, L, 1.0, 2.0)
    assert (lib["cells_x"], lib["n_m"]) == (cells, nm)
    assert lib["ell"] == pytest.approx(ell, rel=1e-15)
