"""The chain kernel's square root: correctly rounded to nearest, bit for bit.

The hit distance of Sec. 3.2 takes sqrt(sigma^2 - c^2) in FP64, and the
trajectories match the oracle's only if that square root is the IEEE one.
The kernel computes it on the integer pipes from an FP32 estimate; these
tests compare it with IEEE sqrt (numpy) and, for inputs whose square root
lies within a tiny fraction of an ulp of a rounding midpoint, with the
rounding decided in exact integer arithmetic.  The host evaluation replaces
the SFU estimate by one perturbed up to 2^-20 (the SFU's error is near
2^-22), so the Newton steps and the final correction are exercised at the
edges of their error budget; the device evaluation is the kernel's own.
"""
import math

import numpy as np
import pytest

from paper_1409_6948_gb300 import ecmc as E

PERTURB = [0.0, 2.0**-22, -2.0**-22, 2.0**-21, -2.0**-21, 2.0**-20, -2.0**-20]


def random_normals(rng, n):
    exp = rng.integers(1, 2047, n, dtype=np.uint64)
    man = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    return ((exp << np.uint64(52)) | man).view(np.float64)


def squares_and_neighbours(rng, n):
    r = rng.integers(1, 1 << 26, n).astype(np.float64)
    k = rng.integers(-400, 400, n)
    sq = np.ldexp(r * r, 2 * k)  # exact squares with exact roots r 2^k
    return np.concatenate([sq, np.nextafter(sq, 0.0), np.nextafter(sq, np.inf)])


def boundary_values():
    out = []
    for c in (1.0, 2.0, 4.0, 0.5, 0.25, 1.0 - 2.0**-53, 2.0**-1022, 2.0**1023):
        v = c
        for _ in range(6):
            out.append(v)
            v = np.nextafter(v, np.inf)
        v = c
        for _ in range(6):
            v = np.nextafter(v, 0.0)
            out.append(v)
    out.append(np.finfo(np.float64).max)
    a = np.array(out, np.float64)
    return a[(a >= 2.0**-1022) & np.isfinite(a)]


def hit_distance_inputs(rng, n):
    # sigma^2 - c^2 for sigma = 1, c uniform in (-1, 1): the kernel's inputs
    db = rng.uniform(-1.0, 1.0, n)
    x = 1.0 - db * db
    return x[x > 0]


def sqrt_mod_pow2(a, n):
    """A root of K^2 = a (mod 2^n) for a = 1 (mod 8), by Hensel lifting."""
    K = 1
    for k in range(3, n):
        if (K * K - a) % (1 << (k + 1)):
            K += 1 << (k - 1)
    assert (K * K - a) % (1 << n) == 0
    return K


def near_midpoint_cases(n_delta=300):
    """x whose sqrt(M 2^52) lies just below or above a midpoint K/2.

    With K odd in [2^53, 2^54) and K^2 = M 2^54 +- delta, sqrt(M 2^52) is
    K/2 -+ about delta / (4K): a few 2^-56 ulp from the midpoint.  Returns
    (x, expected significand as an integer in [2^52, 2^53], exponent E/2).
    """
    xs, want, half = [], [], []
    mod = 1 << 54
    for i in range(n_delta):
        for sign in (+1, -1):
            delta = 8 * i + (1 if sign > 0 else 7)
            target = delta if sign > 0 else mod - delta
            K0 = sqrt_mod_pow2(target, 54)
            for r in {K0 % mod, (-K0) % mod, (K0 + (1 << 53)) % mod, (-K0 + (1 << 53)) % mod}:
                K = r
                if not ((1 << 53) <= K < mod) or K % 2 == 0:
                    continue
                M = (K * K - sign * delta) >> 54
                assert M * mod + sign * delta == K * K
                if not ((1 << 52) <= M < (1 << 54)) or (M >= (1 << 53) and M % 2):
                    continue
                # sqrt(M 2^52) = K/2 - sign * tiny: rounds to (K - sign) / 2
                R = (K - sign) // 2
                E2 = (i % 200) - 100  # E even, E / 2 in [-100, 99]
                xs.append(math.ldexp(float(M), 2 * E2 - 52))
                want.append(R)
                half.append(E2)
    return np.array(xs), want, half


def expected_from_integer(want, half):
    return np.array([math.ldexp(float(R), h - 52) for R, h in zip(want, half)])


def all_inputs(seed=12):
    rng = np.random.default_rng(seed)
    return np.concatenate([random_normals(rng, 200000), squares_and_neighbours(rng, 20000),
                           boundary_values(), hit_distance_inputs(rng, 100000)])


def test_near_midpoint_generator_is_exact():
    x, want, half = near_midpoint_cases(40)
    assert len(x) > 40
    # numpy's IEEE square root agrees with the integer rounding decision
    assert np.array_equal(np.sqrt(x), expected_from_integer(want, half))


@pytest.mark.parametrize("perturb", PERTURB)
def test_host_routine_is_ieee_sqrt(perturb):
    x = all_inputs()
    got = E.sqrt_rn(x, rel_error=perturb)
    ref = np.sqrt(x)
    bad = np.flatnonzero(got.view(np.int64) != ref.view(np.int64))
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], ref[bad[:5]])


@pytest.mark.parametrize("perturb", PERTURB)
def test_host_routine_near_midpoints(perturb):
    x, want, half = near_midpoint_cases()
    got = E.sqrt_rn(x, rel_error=perturb)
    assert np.array_equal(got, expected_from_integer(want, half))


def test_host_routine_rejects_non_normal_inputs():
    x = np.array([0.0, -0.0, -1.0, 2.0**-1074, 2.0**-1023, np.inf, np.nan, 1.0])
    got = E.sqrt_rn(x)
    assert np.all(np.isnan(got[:-1])) and got[-1] == 1.0
    with pytest.raises(E.EcmcError):
        E.sqrt_rn(np.ones(3), rel_error=2.0**-19)


@pytest.mark.gpu
def test_device_routine_is_ieee_sqrt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    xm, want, half = near_midpoint_cases()
    x = np.concatenate([all_inputs(seed=13), xm])
    got = E.sqrt_rn(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = np.sqrt(x)
    bad = np.flatnonzero(got.view(np.int64) != ref.view(np.int64))
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], ref[bad[:5]])
    assert np.array_equal(got[-len(xm):], expected_from_integer(want, half))
    odd = torch.tensor([0.0, -1.0, 2.0**-1074, math.inf, 4.0], dtype=torch.float64).cuda()
    o = E.sqrt_rn(odd).cpu().numpy()
    assert np.all(np.isnan(o[:-1])) and o[-1] == 2.0
