"""Pins of the oracle's variant choices (no GPU): the Jiang-Shu weights (Sec. 2.1), the
Steger-Warming splitting (Sec. 4.4), per-field and local Lax-Friedrichs splitting, and the
reflective wall, each against closed forms, identities of the Euler flux, reductions to the
pinned default scheme, exact equivalences and convergence theory."""
import math

import numpy as np
import pytest

from paper_2004_07954_gb300 import inputs

GAMMA = 1.4


# ------------------------------------------------------------------ Jiang-Shu weights
def test_js_weights_linear_on_quadratics(orc):
    """On quadratic data IS_0 = IS_1 = IS_2, so c_k/(IS_k + eps)^2 normalises to c_k."""
    f = np.array([3.0, 1.5, 0.8, 1.9, 0.2])         # not quadratic: control
    f_q = np.array([(x - 0.3) ** 2 * 2.0 + 1.0 for x in range(-2, 3)])
    r = orc.weno5_parts(f_q, eps=1e-6, kind=orc.W_JS)
    for k, c in enumerate((0.1, 0.6, 0.3)):
        assert r[f"omega{k}"] == pytest.approx(c, abs=1e-15)
    r2 = orc.weno5_parts(f, eps=1e-6, kind=orc.W_JS)
    assert abs(r2["omega1"] - 0.6) > 1e-3


def test_js_weights_eno_at_a_step(orc):
    """A unit step between f_{i+1} and f_{i+2}: only S_0 and S_1 are smooth, the crossing
    sub-stencil S_2 gets weight O(eps^2)."""
    r = orc.weno5_parts([0.0, 0.0, 0.0, 0.0, 1.0], eps=1e-6, kind=orc.W_JS)
    assert r["omega2"] < 1e-11
    assert r["fhat"] == pytest.approx(0.0, abs=1e-11)


def test_js_critical_point_orders(orc):
    """Henrick et al.'s analysis of the Jiang-Shu weights (cited in Sec. 1): fifth order
    where f' != 0, third order at a first-order critical point (approached from above on
    these grids), second order at a second-order one (binary128, eps = 1e-40)."""
    dxs = (0.1, 0.05, 0.025, 0.0125)

    def order(k):
        e = [orc.critical_point_error(k, dx, kind=orc.W_JS, eps=1e-40) for dx in dxs]
        return [math.log2(a / b) for a, b in zip(e[:-1], e[1:])]
    o1, o2, o3 = order(1), order(2), order(3)
    assert min(o1) > 4.9
    assert 3.0 < o2[-1] < 3.4 and o2[0] > o2[1] > o2[2]
    assert all(abs(o - 2.0) < 0.05 for o in o3)


# ------------------------------------------------------------------ Steger-Warming
def _states(nv, seed):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(40):
        rho, p = g.uniform(0.1, 3.0), g.uniform(0.05, 5.0)
        c = math.sqrt(GAMMA * p / rho)
        u = g.uniform(-2.5, 2.5) * c                   # sub- and supersonic both ways
        v = g.uniform(-2.0, 2.0) if nv == 4 else None
        out.append(inputs.cons_from_prim(np.array(rho), u, p, v).ravel())
    return out


@pytest.mark.parametrize("nv", [3, 4])
def test_steger_warming_sums_to_the_flux(orc, nv):
    for U in _states(nv, 1):
        Fp, Fm, F = orc.steger_warming(U, +1), orc.steger_warming(U, -1), orc.normal_flux(U)
        assert np.allclose(Fp + Fm, F, rtol=1e-13, atol=1e-13 * np.abs(F).max())


@pytest.mark.parametrize("nv", [3, 4])
def test_steger_warming_is_the_eigen_split_of_the_homogeneous_flux(orc, nv):
    """The Euler flux is homogeneous of degree one, F = A(U) U, and Steger-Warming is
    F+- = R Lambda+- L U with the state's own eigensystem (the Roe average of a state with
    itself), Lambda+- = diag(max/min(lambda, 0))."""
    for U in _states(nv, 2):
        e = orc.roe_eigen(U, U)
        R, L = e["R"][:nv, :nv], e["L"][:nv, :nv]
        u, c = e["un"], e["c"]
        lam = np.array([u - c, u, u + c] if nv == 3 else [u - c, u, u, u + c])
        for sign in (+1, -1):
            lp = np.maximum(lam, 0.0) if sign > 0 else np.minimum(lam, 0.0)
            want = R @ np.diag(lp) @ L @ U
            got = orc.steger_warming(U, sign)
            assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(orc.normal_flux(U)).max())


def test_steger_warming_supersonic_is_upwind(orc):
    """u > c: F- = 0 exactly and F+ = F; u < -c: the mirror."""
    for u in (2.0, -2.0):
        U = inputs.cons_from_prim(np.array(1.0), u, 1.0).ravel()   # c = sqrt(1.4) < 2
        up, down = (+1, -1) if u > 0 else (-1, +1)
        assert np.all(orc.steger_warming(U, down) == 0.0)
        assert np.allclose(orc.steger_warming(U, up), orc.normal_flux(U), rtol=1e-14)


# ------------------------------------------------------------------ LF speeds
@pytest.mark.parametrize("system,nx,ny", [(1, 64, 1), (2, 20, 16)])
def test_field_speeds_bound_the_lf_speed_exactly(orc, system, nx, ny):
    """max(|u-c|, |u|, |u+c|) = |u| + c, bit for bit, per direction."""
    U = inputs.random_smooth_state(system, nx, ny, seed=3)
    P = orc.problem(system, nx, ny)
    for d in range(2 if system == 2 else 1):
        speeds = [orc.field_speed(P, U, d, k) for k in range(3)]
        assert max(speeds) == orc.max_wavespeed(P, U, d)
        assert speeds[1] < max(speeds)


@pytest.mark.parametrize("system,nx,ny", [(1, 40, 1), (2, 14, 12)])
def test_per_field_lf_with_equal_speeds_is_global_lf(orc, system, nx, ny):
    """Splitting after the projection with alpha_k = alpha for every field equals splitting
    the cells before it (the projection is linear): two independent code paths."""
    U = inputs.random_smooth_state(system, nx, ny, seed=4)
    Pg = orc.problem(system, nx, ny, dx=0.1, dy=0.1, bc_x=orc.PERIODIC, bc_y=orc.OUTFLOW)
    Pf = orc.problem(system, nx, ny, dx=0.1, dy=0.1, bc_x=orc.PERIODIC, bc_y=orc.OUTFLOW, split=orc.S_LF_FIELD)
    ax = orc.max_wavespeed(Pg, U, 0)
    ay = orc.max_wavespeed(Pg, U, 1) if system == 2 else 0.0
    Lg = orc.rhs_speeds(Pg, U, ax, ay)
    Lf = orc.rhs_speeds(Pf, U, ax, ay, fx=(ax,) * 3, fy=(ay,) * 3)
    assert np.abs(Lf - Lg).max() <= 1e-12 * np.abs(Lg).max()
    # and the real per-field speeds are smaller, so the scheme differs
    Lr = orc.rhs(Pf, U)
    assert np.abs(Lr - Lg).max() > 1e-6 * np.abs(Lg).max()


def test_local_lf_with_uniform_speed_is_global_lf(orc):
    """With |u| + c the same in every cell (p proportional to rho, u constant), every
    interface's local speed is the global one up to rounding."""
    n = 64
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x)
    U = inputs.cons_from_prim(rho, 0.4, 1.7 * rho).reshape(3, 1, n)
    Pg = orc.problem(orc.EULER1D, n, dx=1.0 / n, bc_x=orc.PERIODIC)
    Pl = orc.problem(orc.EULER1D, n, dx=1.0 / n, bc_x=orc.PERIODIC, split=orc.S_LLF)
    Lg, Ll = orc.rhs(Pg, U), orc.rhs(Pl, U)
    assert np.abs(Ll - Lg).max() <= 1e-12 * np.abs(Lg).max()
    # a varying |u| + c gives a different (less dissipative) scheme
    V = inputs.random_smooth_state(1, n, 1, seed=5)
    assert np.abs(orc.rhs(Pl, V) - orc.rhs(Pg, V)).max() > 1e-6 * np.abs(orc.rhs(Pg, V)).max()


# ------------------------------------------------------------------ every splitting
SPLITS = ("S_LF_FIELD", "S_LLF", "S_SW")


@pytest.mark.parametrize("split", SPLITS)
def test_splittings_converge_at_fifth_order(orc, split):
    T = 0.5
    errs = []
    for n in (20, 40, 80):
        U0, dx = inputs.entropy_wave_1d(n)
        P = orc.problem(orc.EULER1D, n, dx=dx, bc_x=orc.PERIODIC, split=getattr(orc, split))
        dt = T / math.ceil(T / (0.2 * dx ** (5.0 / 3.0)))
        U, _ = orc.run(P, U0, T, dt)
        exact, _ = inputs.entropy_wave_1d(n, t=T)
        errs.append(np.abs(U[0] - exact[0]).max())
    assert math.log2(errs[0] / errs[1]) > 4.3 and math.log2(errs[1] / errs[2]) > 4.6


@pytest.mark.parametrize("split", SPLITS)
def test_splittings_converge_at_fifth_order_2d(orc, split):
    T = 0.25
    errs = []
    for n in (16, 32):
        U0, dx, dy = inputs.entropy_wave_2d(n, n)
        P = orc.problem(orc.EULER2D, n, n, dx=dx, dy=dy, bc_x=orc.PERIODIC, bc_y=orc.PERIODIC,
                        split=getattr(orc, split))
        dt = T / math.ceil(T / (0.2 * dx ** (5.0 / 3.0)))
        U, _ = orc.run(P, U0, T, dt)
        exact, _, _ = inputs.entropy_wave_2d(n, n, t=T)
        errs.append(np.abs(U[0] - exact[0]).max())
    assert math.log2(errs[0] / errs[1]) > 4.4


@pytest.mark.parametrize("split", SPLITS)
@pytest.mark.parametrize("system,nx,ny", [(1, 50, 1), (2, 12, 10)])
def test_splittings_conserve_and_preserve_free_stream(orc, split, system, nx, ny):
    U0 = inputs.random_smooth_state(system, nx, ny, seed=6)
    P = orc.problem(system, nx, ny, dx=0.1, dy=0.1, bc_x=orc.PERIODIC, bc_y=orc.PERIODIC,
                    split=getattr(orc, split))
    U1, _ = orc.rk3_step(P, U0)
    for k in range(U0.shape[0]):
        assert abs(U1[k].sum() - U0[k].sum()) <= 2e-14 * np.abs(U0[k]).sum()
    prim = inputs.cons_from_prim(np.array(1.3), 0.7, 2.1, -0.4 if system == 2 else None)
    C = np.broadcast_to(prim.reshape(-1, 1, 1), (prim.shape[0], ny, nx)).copy()
    Q = orc.problem(system, nx, ny, dx=0.1, dy=0.1, bc_x=orc.OUTFLOW, bc_y=orc.OUTFLOW, split=getattr(orc, split))
    assert np.abs(orc.rhs(Q, C)).max() <= 1e-13


# ------------------------------------------------------------------ reflective wall
def _mirror_double(U, axis_len, axis):
    """Continue U across its right edge by the mirror image, momentum normal to the wall
    negated (component 1 for x, 2 for y)."""
    M = np.flip(U, axis=axis).copy()
    M[1 if axis == 2 else 2] *= -1.0
    return np.concatenate([U, M], axis=axis)


@pytest.mark.parametrize("split", ["S_LF", "S_SW", "S_LLF"])
def test_reflective_wall_equals_the_mirrored_periodic_problem_1d(orc, split):
    """A grid with reflective walls at both ends has the RHS of the first half of the
    periodic grid of twice the length holding the state and its mirror image: the ghost
    cells coincide, so the RHS agree bit for bit.  Over RK steps the doubled grid's second
    half stays the mirror image only up to rounding (its fluxes come from reversed
    stencils), so the evolved states agree to rounding."""
    n = 60
    U0 = inputs.random_smooth_state(1, n, 1, seed=8)
    P = orc.problem(orc.EULER1D, n, dx=0.1, bc_x=orc.REFLECTIVE, split=getattr(orc, split))
    D0 = _mirror_double(U0, n, 2)
    Q = orc.problem(orc.EULER1D, 2 * n, dx=0.1, bc_x=orc.PERIODIC, split=getattr(orc, split))
    assert np.array_equal(orc.rhs(P, U0), orc.rhs(Q, D0)[:, :, :n])
    U, D = U0.copy(), D0.copy()
    for _ in range(5):
        U, _ = orc.rk3_step(P, U)
        D, _ = orc.rk3_step(Q, D)
    assert np.abs(U - D[:, :, :n]).max() <= 1e-13 * np.abs(U).max()


def test_reflective_wall_equals_the_mirrored_periodic_problem_2d(orc):
    nx, ny = 14, 12
    U0 = inputs.random_smooth_state(2, nx, ny, seed=9)
    P = orc.problem(orc.EULER2D, nx, ny, dx=0.1, dy=0.1, bc_x=orc.OUTFLOW, bc_y=orc.REFLECTIVE)
    D0 = _mirror_double(U0, ny, 1)
    Q = orc.problem(orc.EULER2D, nx, 2 * ny, dx=0.1, dy=0.1, bc_x=orc.OUTFLOW, bc_y=orc.PERIODIC)
    assert np.array_equal(orc.rhs(P, U0), orc.rhs(Q, D0)[:, :ny, :])
    P2 = orc.problem(orc.EULER2D, nx, ny, dx=0.1, dy=0.1, bc_x=orc.REFLECTIVE, bc_y=orc.OUTFLOW)
    D2 = _mirror_double(U0, nx, 2)
    Q2 = orc.problem(orc.EULER2D, 2 * nx, ny, dx=0.1, dy=0.1, bc_x=orc.PERIODIC, bc_y=orc.OUTFLOW)
    assert np.array_equal(orc.rhs(P2, U0), orc.rhs(Q2, D2)[:, :, :nx])


def test_blast_waves_conserve_mass_and_energy_between_walls(orc):
    """Two interacting blast waves (Sec. 4.3.2) between reflective walls: no mass or energy
    crosses a wall."""
    n = 200
    U = inputs.blast_wave_ic(n)
    P = orc.problem(orc.EULER1D, n, dx=1.0 / n, bc_x=orc.REFLECTIVE)
    m0, e0 = U[0].sum(), U[2].sum()
    U, _ = orc.run(P, U, 0.01)
    assert abs(U[0].sum() - m0) <= 1e-13 * m0 and abs(U[2].sum() - e0) <= 1e-13 * e0
    assert np.all(U[0] > 0)
