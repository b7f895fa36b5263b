"""The error bound behind the kernels' LF-speed screen, checked in IEEE single precision.

The screen estimates |u_n| + c from inputs truncated to 20 fraction bits and float
arithmetic with round-to-nearest, and claims a relative error below delta = 1.8e-5 against
the FP64 speed wherever the internal energy is at least an eighth of the total and
rho, E in [2^-30, 2^30), |m| < 2^30.  The exact maximum is then always inside the window
1 - 2^-11 of the running maximum of the estimates (2^-11 > 2 delta / (1 - delta)).  numpy's
float32 operations are IEEE round-to-nearest like the device intrinsics the kernels use.
"""
import numpy as np
import pytest

GAMMA = 1.4
DELTA = 1.8e-5
TAU = 2.0 ** -11


def trunc20(x):
    """float32 with the sign, exponent and leading 20 fraction bits of the float64 x."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    f = (((hi & np.uint32(0x7FFFFFFF)) - np.uint32(896 << 20)) << np.uint32(3)) | (hi & np.uint32(0x80000000))
    return f.view(np.float32)


def in_range(x):
    return (x >= 2.0 ** -30) & (x < 2.0 ** 30)


def estimate_parts(U):
    """(ok, u, v, c) of the single-precision estimate."""
    rho, m, E = U[0], U[1], U[-1]
    n = U[2] if U.shape[0] == 4 else np.zeros_like(rho)
    ok = in_range(rho) & in_range(E) & (np.abs(m) < 2.0 ** 30) & (np.abs(n) < 2.0 ** 30)
    with np.errstate(all="ignore"):
        mf = np.where(np.abs(m) < 2.0 ** -100, np.float32(0), trunc20(m))
        nf = np.where(np.abs(n) < 2.0 ** -100, np.float32(0), trunc20(n))
        rf, Ef = trunc20(rho), trunc20(E)
        r = np.float32(1) / rf
        u, v = mf * r, nf * r
        kin = np.float32(0.5) * (mf * u + nf * v)
        e = Ef - kin
        ok &= e >= np.float32(0.125) * Ef
        c = np.sqrt(np.float32(GAMMA * (GAMMA - 1.0)) * e * r)
    return ok, u, v, c


def estimate(U):
    rho, m, E = U[0], U[1], U[-1]
    n = U[2] if U.shape[0] == 4 else np.zeros_like(rho)
    ok = in_range(rho) & in_range(E) & (np.abs(m) < 2.0 ** 30) & (np.abs(n) < 2.0 ** 30)
    with np.errstate(all="ignore"):
        mf = np.where(np.abs(m) < 2.0 ** -100, np.float32(0), trunc20(m))
        nf = np.where(np.abs(n) < 2.0 ** -100, np.float32(0), trunc20(n))
        rf, Ef = trunc20(rho), trunc20(E)
        r = np.float32(1) / rf
        u, v = mf * r, nf * r
        kin = np.float32(0.5) * (mf * u + nf * v)
        e = Ef - kin
        ok &= e >= np.float32(0.125) * Ef
        gg1 = np.float32(GAMMA * (GAMMA - 1.0))
        c = np.sqrt(gg1 * e * r)
        sx, sy = np.abs(u) + c, np.abs(v) + c
    return ok, sx.astype(np.float64), sy.astype(np.float64)


def exact(U):
    """FP64 speeds in the kernels' (and the oracle's) operation order."""
    rho, m, E = U[0], U[1], U[-1]
    n = U[2] if U.shape[0] == 4 else np.zeros_like(rho)
    u, v = m / rho, n / rho
    kin = (0.5 * rho) * (u * u + v * v)
    p = (GAMMA - 1.0) * (E - kin)
    c = np.sqrt(GAMMA * p / rho)
    return np.abs(u) + c, np.abs(v) + c


def states(seed, count, two_d):
    g = np.random.default_rng(seed)
    lr = g.uniform(-29.0, 29.0, size=count) * np.log(2.0)
    rho = np.exp(lr)
    # pressures spread so that e/E covers [1/8 - margin, 1]; velocities of both signs
    p = rho * np.exp(g.uniform(-20.0, 20.0, size=count))
    p = np.minimum(p, 2.0 ** 28)
    c = np.sqrt(GAMMA * p / rho)
    mach = g.choice([0.0, 1e-20, 0.1, 1.0, 3.0, 4.9, 5.0, 5.1], size=count) * g.uniform(0.5, 1.0, size=count)
    ang = g.uniform(0, 2 * np.pi, size=count)
    u = mach * c * np.cos(ang)
    v = mach * c * np.sin(ang) if two_d else np.zeros(count)
    E = p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v)
    rows = [rho, rho * u] + ([rho * v] if two_d else []) + [E]
    return np.stack(rows)


@pytest.mark.parametrize("two_d", [False, True])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_estimate_within_delta(two_d, seed):
    U = states(seed, 400_000, two_d)
    ok, ex, ey = estimate(U)
    sx, sy = exact(U)
    assert ok.mean() > 0.3                    # the bound is exercised on many states
    rel = np.abs(ex - sx)[ok] / sx[ok]
    assert rel.max() <= DELTA, rel.max()
    if two_d:
        rel_y = np.abs(ey - sy)[ok] / sy[ok]
        assert rel_y.max() <= DELTA, rel_y.max()
    # every screened state is admissible in FP64: p > 0, finite speeds
    rho, m, E = U[0], U[1], U[-1]
    kin = (0.5 * rho) * ((m / rho) ** 2 + ((U[2] / rho) ** 2 if two_d else 0.0))
    assert np.all(((GAMMA - 1.0) * (E - kin))[ok] > 0.0)
    assert np.all(np.isfinite(sx[ok]))


@pytest.mark.parametrize("two_d", [False, True])
def test_field_estimates_within_delta_of_the_lf_speed(two_d):
    """Per-field speeds |u-c|, |u|, |u+c|: each estimate is within delta (|u| + c) of the
    FP64 value (the window of the per-field screen is relative to the LF speed)."""
    U = states(11, 400_000, two_d)
    ok, uf, vf, cf = estimate_parts(U)
    rho, m, E = U[0], U[1], U[-1]
    u = m / rho
    v = U[2] / rho if two_d else np.zeros_like(u)
    kin = (0.5 * rho) * (u * u + v * v)
    c = np.sqrt(GAMMA * ((GAMMA - 1.0) * (E - kin)) / rho)
    with np.errstate(all="ignore"):
        for w, wf in ((u, uf), (v, vf)):
            s = np.abs(w) + c
            for exact, est in ((np.abs(w - c), np.abs(wf - cf)), (np.abs(w), np.abs(wf)), (np.abs(w + c), np.abs(wf + cf))):
                err = np.abs(est.astype(np.float64) - exact)[ok] / s[ok]
                assert err.max() <= DELTA, err.max()


def test_window_covers_twice_delta():
    assert TAU >= 2 * DELTA / (1 - DELTA)
    assert np.float32(1.0 - TAU) == np.float32(1.0) - np.float32(1.0 / 2048.0)


def test_truncation_error_below_2_pow_20():
    g = np.random.default_rng(9)
    x = np.exp(g.uniform(-80, 80, size=200_000)) * g.choice([-1.0, 1.0], size=200_000)
    t = trunc20(x).astype(np.float64)
    rel = np.abs(t - x) / np.abs(x)
    assert rel.max() < 2.0 ** -20
    assert np.all(np.abs(t) <= np.abs(x)) and np.all(np.sign(t) == np.sign(x))


def test_unscreened_cases():
    """States outside the proven range carry no estimate."""
    cols = [
        (1e-10, 0.0, 2.5),        # rho below 2^-30
        (2e9, 0.0, 2.5e9),        # rho and E above 2^30
        (1.0, 0.0, 2e9),          # E above 2^30
        (1.0, 2e9, 3e18),         # |m| above 2^30
        (1.0, 10.0, 51.0),        # kinetic energy 50/51 of the total
        (1.0, np.nan, 2.5),       # NaN momentum
        (-1.0, 0.0, 2.5),         # negative density
        (1.0, 0.0, -2.5),         # negative energy
    ]
    ok, _, _ = estimate(np.array(cols).T.copy())
    assert not ok.any()
    ok, _, _ = estimate(np.array([(1.0, 0.0, 2.5), (1.0, 1.0, 3.0)]).T.copy())
    assert ok.all()
