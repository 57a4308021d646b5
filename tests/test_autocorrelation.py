"""Pins of the autocorrelation time (Sec. 2, eq. tau) on both sides: the
oracle's orc_autocorrelation_time and the library's host-side
ecmc_autocorrelation_time (no GPU needed).

C(dt) = Re <Psi*(t) Psi(t+dt)> / <|Psi|^2>, tau = its 1/e lag interpolated
linearly.  Closed forms: a rotating complex AR(1) process z_{t+1} = a e^{i w}
z_t + noise has C(dt) = a^dt cos(w dt); a pure rotation has C(dt) = cos(w dt)
exactly.  Dropping the conjugate or the real part, or normalising by the wrong
number of pairs, fails one of them.
"""
import math

import numpy as np
import pytest

import oracle


def rotating_ar1(a, w, n, seed):
    rng = np.random.default_rng(seed)
    noise = rng.normal(size=n) + 1j * rng.normal(size=n)
    z = np.empty(n, complex)
    z[0] = noise[0] / math.sqrt(1 - a * a)
    f = a * complex(math.cos(w), math.sin(w))
    for t in range(1, n):
        z[t] = f * z[t - 1] + noise[t]
    return z


def first_crossing(a, w):
    # smallest real dt with a^dt cos(w dt) = 1/e, by bisection on the first
    # bracket of the integer lags
    f = lambda d: a**d * math.cos(w * d) - math.exp(-1.0)  # noqa: E731
    d = 0
    while f(d + 1) >= 0:
        d += 1
    lo, hi = float(d), float(d + 1)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) >= 0 else (lo, mid)
    return lo


def library_tau():
    P = pytest.importorskip("paper_1409_6948_gb300")
    try:
        P.load()
    except Exception as e:  # noqa: BLE001
        pytest.skip("library not built: %s" % e)
    from paper_1409_6948_gb300.ecmc import autocorrelation_time
    return autocorrelation_time


@pytest.mark.parametrize("side", ["oracle", "library"])
@pytest.mark.parametrize("tau0,w", [(12.5, 0.0), (20.0, 0.05)])
def test_rotating_ar1(side, tau0, w):
    a = math.exp(-1.0 / tau0)
    z = rotating_ar1(a, w, 200000, 7)
    fn = oracle.autocorrelation_time if side == "oracle" else library_tau()
    tau, c = fn(z, 100)
    for d in (1, 5, 10, 20):
        assert abs(c[d] - a**d * math.cos(w * d)) < 0.02, (d, c[d])
    want = first_crossing(a, w)
    assert abs(tau - want) < 0.05 * want, (tau, want)


@pytest.mark.parametrize("side", ["oracle", "library"])
def test_pure_rotation_is_exact(side):
    w, n, lag = 0.11, 4000, 40
    t = np.arange(n)
    z = 1.7 * np.exp(1j * w * t)
    fn = oracle.autocorrelation_time if side == "oracle" else library_tau()
    tau, c = fn(z, lag)
    assert np.allclose(c, np.cos(w * np.arange(lag + 1)), atol=1e-12, rtol=0)
    d = int(np.flatnonzero(c < math.exp(-1.0))[0])
    assert d - 1 <= tau <= d
    assert tau == pytest.approx((d - 1) + (c[d - 1] - math.exp(-1.0)) / (c[d - 1] - c[d]),
                                rel=1e-14)


def test_no_crossing_gives_infinity_and_the_two_sides_agree():
    z = rotating_ar1(math.exp(-1.0 / 500.0), 0.0, 3000, 3)
    ft = library_tau()
    t_lib, c_lib = ft(z, 50)
    t_orc, c_orc = oracle.autocorrelation_time(z, 50)
    assert math.isinf(t_lib) and math.isinf(t_orc)
    z = rotating_ar1(math.exp(-1.0 / 8.0), 0.3, 5000, 4)
    t_lib, c_lib = ft(z, 60)
    t_orc, c_orc = oracle.autocorrelation_time(z, 60)
    assert np.allclose(c_lib, c_orc, rtol=1e-13, atol=1e-15)
    assert t_lib == pytest.approx(t_orc, rel=1e-13)


@pytest.mark.parametrize("side", ["oracle", "library"])
def test_replicas_average_the_closed_form(side):
    # 16 independent AR(1) series of 20,000 samples: the replica average has
    # the single series' C(dt) = a^dt cos(w dt); the same data as one long
    # series would mix the replicas' ends
    a, w = math.exp(-1.0 / 10.0), 0.07
    z = np.stack([rotating_ar1(a, w, 20000, 100 + r) for r in range(16)], axis=1)
    fn = oracle.autocorrelation_time if side == "oracle" else library_tau()
    tau, c = fn(z, 60)
    for d in (1, 5, 10, 20):
        assert abs(c[d] - a**d * math.cos(w * d)) < 0.015, (d, c[d])
    want = first_crossing(a, w)
    assert abs(tau - want) < 0.04 * want, (tau, want)
    # replicas of identical series: the average equals the single series
    z1 = rotating_ar1(a, w, 5000, 7)
    t1, c1 = fn(z1, 30)
    t4, c4 = fn(np.stack([z1] * 4, axis=1), 30)
    assert np.allclose(c1, c4, rtol=1e-12) and t1 == pytest.approx(t4, rel=1e-12)


def test_library_rejects_bad_arguments():
    library_tau()
    import ctypes as C
    from paper_1409_6948_gb300 import ecmc as E
    lib = E.load()
    buf = np.ones(20)
    tau = C.c_double()
    assert lib.ecmc_autocorrelation_time(buf.ctypes.data, 1, 1, 0, C.byref(tau),
                                         None) == E.ERR_ARG
    assert lib.ecmc_autocorrelation_time(buf.ctypes.data, 10, 1, 10, C.byref(tau),
                                         None) == E.ERR_ARG
    assert lib.ecmc_autocorrelation_time(buf.ctypes.data, 10, 0, 2, C.byref(tau),
                                         None) == E.ERR_ARG
    assert lib.ecmc_autocorrelation_time(None, 10, 1, 2, C.byref(tau), None) == E.ERR_ARG
    zero = np.zeros(20)
    assert lib.ecmc_autocorrelation_time(zero.ctypes.data, 10, 1, 2, C.byref(tau),
                                         None) == E.ERR_ARG
