"""Pins of the CPU oracle's reconstruction against numbers the paper prints and against
closed forms of the mathematics (no GPU)."""
import math

import numpy as np
import pytest

from conftest import read_golden

EPS = 1e-40


# ------------------------------------------------------------------ Sec. 3, coefficient table
def test_table1_step_coefficients(orc):
    """A single jump of height h between f_{i+k-1} and f_{i+k} gives tau5 = c5 h^2 and
    tau8 = c8 h^2 with the coefficients the paper tabulates."""
    for k, t5n, t5d, t8 in read_golden("table1_step_coefficients.txt"):
        for h in (1.0, -3.5, 0.25):
            pos = int(k) + 2          # first stencil index on the high side of the jump
            f = np.array([0.0 if s < pos else h for s in range(5)])
            p = orc.weno5_parts(f)
            assert p["tau5"] == pytest.approx(t5n / t5d * h * h, rel=1e-14)
            assert p["tau8"] == pytest.approx(t8 * h * h, rel=1e-14)


# ------------------------------------------------------------------ Sec. 3, worked example
def _u0_single(x):
    # Eq. (single); the printed u0(0) = 0 is the left branch's value at x = 0.
    v = -math.sin(math.pi * x) - 0.5 * x ** 3
    return v + 1.0 if x > 1e-12 else v


def test_table2_worked_example(orc):
    dx = 0.02
    for xi, u, t5, t8, R, Rp in read_golden("table2_worked_example.txt"):
        i = round(xi / dx)
        f = [_u0_single((i + s) * dx) for s in range(-2, 3)]
        p = orc.weno5_parts(f)
        IS0, IS2, C = p["IS0"], p["IS2"], p["C"]
        big, small = (IS0, IS2) if IS0 >= IS2 else (IS2, IS0)
        r = (1 + p["tau5"] / (big + EPS)) / (1 + p["tau5"] / (small + EPS))
        rp = (C + p["tau8"] / (big + EPS)) / (C + p["tau8"] / (small + EPS))
        assert abs(_u0_single(i * dx) - u) <= 0.6e-4 * max(1.0, abs(u)) + 1e-12
        assert p["tau5"] == pytest.approx(t5, rel=2e-3)
        assert p["tau8"] == pytest.approx(t8, rel=2e-3)
        # rows where IS_0 and IS_2 agree to rounding print either sign: compare |R|, |R'|
        assert r == pytest.approx(abs(R), rel=2e-3)
        assert rp == pytest.approx(abs(Rp), rel=2e-3)


# ------------------------------------------------------------------ Sec. 4.1, critical points
TABLE3 = read_golden("table3_critical_point.txt")


@pytest.mark.parametrize("row", TABLE3, ids=[f"k{int(r[0])}-j{int(r[1])}" for r in TABLE3])
def test_table3_quad_precision(orc, row):
    """All 24 WENO-ZN and 24 WENO-Z (q=1) cells in binary128 arithmetic."""
    k, j, z_err, _za_err, zn_err = row
    dx = 0.025 / 2 ** int(j)
    assert orc.critical_point_error(int(k), dx, orc.W_ZN, EPS, quad=True) == pytest.approx(zn_err, rel=1e-5)
    assert orc.critical_point_error(int(k), dx, orc.W_Z, EPS, quad=True) == pytest.approx(z_err, rel=1e-5)


# rows whose error sits above FP64 round-off of the difference quotient
FP64_ROWS = {1: range(0, 2), 2: range(0, 5), 3: range(0, 8)}


@pytest.mark.parametrize("k", [1, 2, 3])
def test_table3_double_precision_rows(orc, k):
    for row in TABLE3:
        if int(row[0]) != k or int(row[1]) not in FP64_ROWS[k]:
            continue
        dx = 0.025 / 2 ** int(row[1])
        assert orc.critical_point_error(k, dx, orc.W_ZN, EPS, quad=False) == pytest.approx(row[4], rel=1e-4)


def test_table3_orders(orc):
    """Orders the paper states: 5 at a first-order critical point, about 4 at a second-order
    one for WENO-ZN; about 4 and about 2 for WENO-Z (q=1)."""
    def order(k, kind, j):
        e0 = orc.critical_point_error(k, 0.025 / 2 ** j, kind, EPS, quad=True)
        e1 = orc.critical_point_error(k, 0.025 / 2 ** (j + 1), kind, EPS, quad=True)
        return math.log2(e0 / e1)
    assert order(2, orc.W_ZN, 6) == pytest.approx(5.0, abs=0.01)
    assert order(3, orc.W_ZN, 6) == pytest.approx(3.98, abs=0.02)
    assert order(2, orc.W_Z, 6) == pytest.approx(4.003, abs=0.01)
    assert order(3, orc.W_Z, 6) == pytest.approx(2.06, abs=0.02)


# ------------------------------------------------------------------ Sec. 3 property analysis
def test_weights_order_at_critical_points(orc):
    """Eq. (C1)/(C): max_k |omega_k - c_k| at x = 0 on x^k e^x falls like dx^14, dx^7, dx^4
    for k = 1, 2, 3 (all at least the sufficient dx^3 of Eq. (10))."""
    c = np.array([0.1, 0.6, 0.3])
    for k, lo in ((1, 13.5), (2, 6.5), (3, 3.5)):
        devs = []
        for j in (2, 3):
            dx = 0.025 / 2 ** j
            x = dx * np.arange(-2, 3)
            f = x ** k * np.exp(x)
            p = orc.weno5_parts(f)
            devs.append(max(abs(p[f"omega{m}"] - c[m]) for m in range(3)))
        if devs[1] == 0.0:
            continue           # already at round-off
        assert math.log2(devs[0] / devs[1]) >= lo


def test_constant_data_gives_C_equal_A_and_linear_weights(orc):
    p = orc.weno5_parts([2.5] * 5)
    assert p["IS0"] == p["IS1"] == p["IS2"] == 0.0
    assert p["tau5"] == 0.0 and p["tau8"] == 0.0
    assert p["C"] == pytest.approx(10.0, rel=1e-15)
    assert [p["omega0"], p["omega1"], p["omega2"]] == pytest.approx([0.1, 0.6, 0.3], rel=1e-15)
    assert p["fhat"] == pytest.approx(2.5, rel=1e-15)


@pytest.mark.parametrize("coef", [(1.0, -2.0, 3.0, 1.0), (0.5, 4.0, -1.0, -2.0), (-3.0, 0.0, 0.0, 2.0)])
def test_cubic_data_linear_weights_and_exact_derivative(orc, coef):
    """On cubic samples tau8 = 0 exactly (integer data), so alpha_k = c_k C and omega = c;
    the linear fifth-order scheme then differentiates polynomials of degree <= 4 exactly:
    (f^_{i+1/2} - f^_{i-1/2}) / dx = f'(x_i)."""
    a0, a1, a2, a3 = coef
    f = lambda x: a0 + a1 * x + a2 * x * x + a3 * x ** 3
    df = lambda x: a1 + 2 * a2 * x + 3 * a3 * x * x
    for xi in (-3, 0, 2, 7):
        xs = np.arange(xi - 3, xi + 3, dtype=np.float64)       # x_{i-3} .. x_{i+2}
        vals = f(xs)
        pr = orc.weno5_parts(vals[1:6])
        pl = orc.weno5_parts(vals[0:5])
        assert pr["tau8"] == 0.0
        assert [pr["omega0"], pr["omega1"], pr["omega2"]] == pytest.approx([0.1, 0.6, 0.3], rel=1e-14)
        d = pr["fhat"] - pl["fhat"]
        assert d == pytest.approx(df(xi), rel=1e-12, abs=1e-11)


def test_quadratic_data_equal_indicators(orc):
    """On quadratic samples IS_0 = IS_1 = IS_2 (both of their differences are the same),
    hence tau5 = 0."""
    x = np.arange(-2, 3, dtype=np.float64)
    p = orc.weno5_parts(3 * x * x - x + 4)
    assert p["IS0"] == p["IS1"] == p["IS2"]
    assert p["tau5"] == 0.0


@pytest.mark.parametrize("pos", [1, 2, 3, 4])
def test_step_crossing_substencils_get_no_weight(orc, pos):
    """Property (2): with a pure jump the sub-stencils that straddle it get weight
    < 1e-30; a smooth (constant) sub-stencil keeps almost all of it."""
    f = np.array([0.0 if s < pos else 1.0 for s in range(5)])
    p = orc.weno5_parts(f)
    assert p["C"] < 1e-2
    # sub-stencil k spans indices k..k+2; it crosses the jump iff k < pos <= k+2
    for k in range(3):
        crosses = k < pos <= k + 2
        if crosses:
            assert p[f"omega{k}"] < 1e-30
    smooth = [k for k in range(3) if not (k < pos <= k + 2)]
    assert sum(p[f"omega{k}"] for k in smooth) == pytest.approx(1.0, abs=1e-30)


@pytest.mark.parametrize("lam,rel", [(2.0 ** 7, 0.0), (2.0 ** -7, 0.0), (-8.0, 0.0), (1e2, 1e-9), (1e-2, 1e-9)])
def test_self_similarity(orc, lam, rel):
    """Scaling the data by lam scales the flux by lam (eps = 1e-40 is negligible): the
    dimensional consistency the paper asks of a weight function (Sec. 2.3, Sec. 4.2).
    Power-of-two factors scale every intermediate exactly; other factors perturb the inputs
    by one rounding, which the nonlinear weights may amplify."""
    g = np.random.default_rng(3)
    for _ in range(50):
        f = g.normal(size=5) * g.choice([1e-3, 1.0, 1e3])
        got = orc.weno5_parts(lam * f)["fhat"]
        want = lam * orc.weno5_parts(f)["fhat"]
        if rel == 0.0:
            assert got == want
        else:
            assert got == pytest.approx(want, rel=rel)


def test_minus_side_is_mirror_of_plus_side(orc):
    g = np.random.default_rng(5)
    n = 37
    f = g.normal(size=n + 6)
    plus = orc.reconstruct(f, +1)
    minus_mirror = orc.reconstruct(f[::-1].copy(), -1)[::-1]
    assert np.array_equal(plus, minus_mirror)


def test_weights_are_convex(orc):
    g = np.random.default_rng(11)
    for _ in range(200):
        f = g.normal(size=5) * 10 ** g.uniform(-3, 3)
        p = orc.weno5_parts(f)
        w = np.array([p["omega0"], p["omega1"], p["omega2"]])
        assert np.all(w >= 0) and w.sum() == pytest.approx(1.0, rel=1e-14)
        q = np.array([p["q0"], p["q1"], p["q2"]])
        assert q.min() - 1e-12 * abs(q).max() <= p["fhat"] <= q.max() + 1e-12 * abs(q).max()


def test_substencil_fluxes_exact_on_quadratics(orc):
    """Each q_k of Eq. (4) is the third-order reconstruction: exact at x_{i+1/2} for the
    cell-average data of a quadratic."""
    # cell averages of h(x) = x^2 over [j-1/2, j+1/2] are j^2 + 1/12 (dx = 1)
    j = np.arange(-2, 3, dtype=np.float64)
    avg = j * j + 1.0 / 12.0
    p = orc.weno5_parts(avg)
    for k in range(3):
        assert p[f"q{k}"] == pytest.approx(0.25, rel=1e-14)     # h(1/2)


def test_reconstruct_matches_pointwise_parts(orc):
    g = np.random.default_rng(9)
    n = 23
    f = g.normal(size=n + 6)
    out = orc.reconstruct(f, +1)
    for j in range(n + 1):
        assert out[j] == orc.weno5_parts(f[j:j + 5])["fhat"]


def test_ghost_fill_line(orc):
    n = 9
    vals = np.arange(10.0, 10.0 + n)
    pad = np.zeros(n + 6)
    pad[3:n + 3] = vals
    per = orc.fill_ghosts_line(pad, orc.PERIODIC)
    out = orc.fill_ghosts_line(pad, orc.OUTFLOW)
    for g in range(1, 4):
        assert per[3 - g] == vals[n - g] and per[n + 2 + g] == vals[g - 1]
        assert out[3 - g] == vals[0] and out[n + 2 + g] == vals[n - 1]


# ------------------------------------------------------------------ binary128 line reconstruction
@pytest.mark.parametrize("kind,eps", [(0, EPS), (1, EPS), (3, 1e-6)])
def test_quad_reconstruction_equals_double_on_ordinary_data(orc, kind, eps):
    """The binary128 evaluation (the range reference) rounds to the double evaluation on data
    where the latter stays in range."""
    g = np.random.default_rng(3 + kind)
    f = g.normal(size=506)
    f[g.random(506) < 0.1] += 5.0
    for side in (1, -1):
        d = orc.reconstruct(f, side, eps=eps, kind=kind)
        q = orc.reconstruct_quad(f, side, eps=eps, kind=kind)
        assert np.abs(d - q).max() <= 1e-13 * np.abs(f).max()


@pytest.mark.parametrize("k", [150, 300, 433])
def test_quad_reconstruction_homogeneous_in_data_and_eps(orc, k):
    """Eq. (function) and Eq. (new) are homogeneous: f -> s f with eps -> s^2 eps scales every
    IS_k, tau5, tau8 by s^2 and leaves C and the weights unchanged, so f^(s f; eps) =
    s f^(f; eps / s^2) exactly for a power of two s; the binary128 evaluation keeps this at
    scales where the double one overflows."""
    s = 2.0 ** k
    g = np.random.default_rng(k)
    f = g.normal(size=206)
    f[g.random(206) < 0.1] += 5.0
    for side in (1, -1):
        big = orc.reconstruct_quad(f * s, side, eps=EPS)
        small = orc.reconstruct_quad(f, side, eps=EPS / s ** 2)
        assert np.all(np.isfinite(big))
        assert np.abs(big - small * s).max() <= 1e-15 * np.abs(f * s).max()


def test_quad_reconstruction_linear_limit_at_equal_large_indicators(orc):
    """Where tau5 = |IS_0 - IS_2| = 0 and the indicators are huge, C = A ((IS_0 + IS_2 + eps)
    / eps)^2 dwarfs tau8 / (IS_k + eps) and the weights are the linear ones to far below
    double rounding: the plain double evaluation overflows C there (NaN), the binary128 one
    gives the linear scheme's flux."""
    f = np.full(26, 0.7)
    f[12] = -2.0                                       # IS_0 = IS_2 at the interface beside the spike
    f *= 1e100
    lin = orc.reconstruct(f, 1, kind=2)
    q = orc.reconstruct_quad(f, 1)
    d = orc.reconstruct(f, 1)
    bad = ~np.isfinite(d)
    assert bad.any()                                   # the double evaluation's own overflow
    assert np.abs(q[bad] - lin[bad]).max() <= 1e-15 * np.abs(f).max()
    assert np.abs(q[~bad] - d[~bad]).max() <= 1e-13 * np.abs(f).max()
