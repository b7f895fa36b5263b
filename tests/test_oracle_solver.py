"""Pins of the CPU oracle's solver (flux splitting, characteristic fields, RHS, SSP-RK3)
against exact solutions, closed forms and invariants (no GPU)."""
import math

import numpy as np
import pytest

from paper_2004_07954_gb300 import inputs

GAMMA = 1.4


def _prim_state(rho, u, p, v=None):
    return inputs.cons_from_prim(np.array(rho), u, p, v)


# ------------------------------------------------------------------ characteristic fields
def _jacobian_fd(orc, U, h=1e-6):
    nv = U.shape[0]
    J = np.zeros((nv, nv))
    for m in range(nv):
        e = np.zeros(nv)
        e[m] = h * max(1.0, abs(U[m]))
        J[:, m] = (orc.normal_flux(U + e) - orc.normal_flux(U - e)) / (2 * e[m])
    return J


@pytest.mark.parametrize("nv", [3, 4])
def test_left_right_eigenvectors(orc, nv):
    """R L = I, and L J R = diag(u-c, u, [u,] u+c) with J the flux Jacobian taken by central
    differences of the oracle's flux (an independent route to the eigen-system)."""
    g = np.random.default_rng(1)
    for _ in range(10):
        rho, u, v, p = g.uniform(0.3, 3), g.uniform(-2, 2), g.uniform(-2, 2), g.uniform(0.2, 5)
        U = _prim_state(rho, u, p, v if nv == 4 else None)
        e = orc.roe_eigen(U, U)
        c = math.sqrt(GAMMA * p / rho)
        assert e["c"] == pytest.approx(c, rel=1e-13)
        assert e["R"] @ e["L"] == pytest.approx(np.eye(nv), abs=1e-13)
        lam = [u - c, u, u + c] if nv == 3 else [u - c, u, u, u + c]
        D = e["L"] @ _jacobian_fd(orc, U) @ e["R"]
        assert D == pytest.approx(np.diag(lam), abs=2e-7 * max(1.0, abs(u) + c))


@pytest.mark.parametrize("nv", [3, 4])
def test_roe_property(orc, nv):
    """The Roe average satisfies F(U_R) - F(U_L) = R Lambda L (U_R - U_L) exactly (Roe's
    defining property), which pins the averaging as well as the eigenvectors."""
    g = np.random.default_rng(2)
    for _ in range(20):
        sl = [g.uniform(0.2, 4), g.uniform(-2, 2), g.uniform(0.1, 8), g.uniform(-2, 2)]
        sr = [g.uniform(0.2, 4), g.uniform(-2, 2), g.uniform(0.1, 8), g.uniform(-2, 2)]
        UL = _prim_state(sl[0], sl[1], sl[2], sl[3] if nv == 4 else None)
        UR = _prim_state(sr[0], sr[1], sr[2], sr[3] if nv == 4 else None)
        e = orc.roe_eigen(UL, UR)
        u, c = e["un"], e["c"]
        lam = np.array([u - c, u, u + c] if nv == 3 else [u - c, u, u, u + c])
        A = e["R"] @ np.diag(lam) @ e["L"]
        dF = orc.normal_flux(UR) - orc.normal_flux(UL)
        assert A @ (UR - UL) == pytest.approx(dF, rel=1e-11, abs=1e-11 * np.abs(dF).max())


# ------------------------------------------------------------------ RK3
@pytest.mark.parametrize("z", [-0.5, -1.0, -2.5, 0.3, 1j * 0.0 - 1.7])
def test_rk3_stability_polynomial(orc, z):
    """Shu-Osher SSP-RK3 on u' = lam u multiplies by 1 + z + z^2/2 + z^3/6, z = lam dt."""
    z = float(np.real(z))
    got = orc.rk3_linear(z / 0.1, 0.1, 1.0)
    assert got == pytest.approx(1 + z + z * z / 2 + z ** 3 / 6, rel=1e-15, abs=1e-15)


# ------------------------------------------------------------------ advection
def _adv_problem(orc, n, kind=0):
    _, dx = inputs.advection_grid(n)
    return orc.problem(orc.ADV1D, n, 1, dx=dx, bc_x=orc.PERIODIC, weights=kind)


def _adv_errors(orc, n, which, kind=0, T=2.0):
    P = _adv_problem(orc, n, kind)
    dt, steps = inputs.advection_dt(n, T)
    U, nsteps = orc.run(P, inputs.advection_ic(n, which), T, dt)
    assert nsteps == steps
    err = (U - inputs.advection_exact(n, which, T)).ravel()
    return np.abs(err).mean(), np.abs(err).max()


@pytest.mark.parametrize("which", ["sin", "critical"])
def test_advection_fifth_order(orc, which):
    """Fifth-order L1 and Linf convergence on smooth periodic advection, also with a
    first-order critical point in the profile; ZN within 10 % of the linear upwind scheme."""
    ns = (40, 80, 160)
    errs = [_adv_errors(orc, n, which) for n in ns]
    for (l1a, lia), (l1b, lib) in zip(errs[1:], errs[2:]):
        assert 4.7 <= math.log2(l1a / l1b) <= 5.3
        assert 4.7 <= math.log2(lia / lib) <= 5.3
    lin = _adv_errors(orc, 160, which, kind=2)
    assert errs[-1][0] <= 1.1 * lin[0] and errs[-1][1] <= 1.1 * lin[1]


def test_advection_conservation_periodic(orc):
    n = 64
    P = _adv_problem(orc, n)
    U0 = inputs.random_smooth_state(0, n, 1, seed=4)
    U1, _ = orc.rk3_step(P, U0, 0.3 * P.dx)
    assert abs(U1.sum() - U0.sum()) <= 1e-13 * np.abs(U0).sum()


# ------------------------------------------------------------------ Euler
def _euler_periodic(orc, system, nx, ny, dx, dy=1.0):
    return orc.problem(system, nx, ny, dx=dx, dy=dy, bc_x=orc.PERIODIC, bc_y=orc.PERIODIC)


def test_euler1d_entropy_wave_fifth_order(orc):
    """A density sine carried by u = 1 at p = 1 is an exact Euler solution; the scheme
    converges to it at fifth order (time step small enough that RK3 error stays below)."""
    T = 0.5
    errs = []
    for n in (20, 40, 80):
        U0, dx = inputs.entropy_wave_1d(n)
        P = _euler_periodic(orc, orc.EULER1D, n, 1, dx)
        dt = T / math.ceil(T / (0.2 * dx ** (5.0 / 3.0)))
        U, _ = orc.run(P, U0, T, dt)
        exact, _ = inputs.entropy_wave_1d(n, t=T)
        errs.append(np.abs(U[0] - exact[0]).max())
    assert math.log2(errs[0] / errs[1]) > 4.4 and math.log2(errs[1] / errs[2]) > 4.7


def test_euler2d_entropy_wave_fifth_order(orc):
    """Same exact solution in 2D moving along (1, 0.5): exercises both sweeps and the
    state permutation of the y-sweep."""
    T = 0.25
    errs = []
    for n in (16, 32):
        U0, dx, dy = inputs.entropy_wave_2d(n, n)
        P = _euler_periodic(orc, orc.EULER2D, n, n, dx, dy)
        dt = T / math.ceil(T / (0.2 * dx ** (5.0 / 3.0)))
        U, _ = orc.run(P, U0, T, dt)
        exact, _, _ = inputs.entropy_wave_2d(n, n, t=T)
        errs.append(np.abs(U[0] - exact[0]).max())
    assert math.log2(errs[0] / errs[1]) > 4.5


@pytest.mark.parametrize("system,nx,ny", [(1, 50, 1), (2, 12, 10)])
def test_euler_conservation_periodic(orc, system, nx, ny):
    U0 = inputs.random_smooth_state(system, nx, ny, seed=6)
    P = _euler_periodic(orc, system, nx, ny, 0.1, 0.1)
    U1, dt = orc.rk3_step(P, U0)
    for k in range(U0.shape[0]):
        assert abs(U1[k].sum() - U0[k].sum()) <= 2e-14 * np.abs(U0[k]).sum()


@pytest.mark.parametrize("system,nx,ny", [(1, 40, 1), (2, 9, 11)])
def test_free_stream_preservation(orc, system, nx, ny):
    rho, u, v, p = 1.3, 0.7, -0.4, 2.1
    prim = _prim_state(rho, u, p, v if system == 2 else None)
    U = np.broadcast_to(prim.reshape(-1, 1, 1), (prim.shape[0], ny, nx)).copy()
    for bc in (0, 1):
        P = orc.problem(system, nx, ny, dx=0.1, dy=0.1, bc_x=bc, bc_y=bc)
        L = orc.rhs(P, U)
        assert np.abs(L).max() <= 1e-13


def test_euler1d_outflow_flux_balance(orc):
    """With constant states next to both outflow boundaries, the discrete RHS sums to the
    boundary flux difference: sum_i L_i dx = F(U_left) - F(U_right)."""
    n = 60
    U = inputs.random_smooth_state(1, n, 1, seed=8)
    U[:, :, :5] = U[:, :, :1].copy()
    U[:, :, -5:] = U[:, :, -1:].copy()
    P = orc.problem(orc.EULER1D, n, 1, dx=0.05, bc_x=orc.OUTFLOW)
    L = orc.rhs(P, U)
    want = orc.normal_flux(U[:, 0, 0]) - orc.normal_flux(U[:, 0, -1])
    assert (L[:, 0, :].sum(axis=1) * 0.05) == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_euler1d_mirror_symmetry(orc):
    """x -> -x with u -> -u maps the solution onto its mirror image."""
    n = 80
    U = inputs.euler1d_ic(n, seed=3)
    M = U[:, :, ::-1].copy()
    M[1] = -M[1]
    P = orc.problem(orc.EULER1D, n, 1, dx=10.0 / n, bc_x=orc.OUTFLOW)
    for _ in range(20):
        U, dt1 = orc.rk3_step(P, U)
        M, dt2 = orc.rk3_step(P, M)
        assert dt1 == pytest.approx(dt2, rel=1e-14)
    Mb = M[:, :, ::-1].copy()
    Mb[1] = -Mb[1]
    assert np.abs(U - Mb).max() <= 1e-12 * np.abs(U).max()


def test_euler2d_transpose_symmetry(orc):
    """Swapping x and y together with u and v maps the 2D solution onto its transpose."""
    n = 16
    U = inputs.euler2d_ic(n, n, seed=1)
    T = np.stack([U[0].T, U[2].T, U[1].T, U[3].T]).copy()
    P = orc.problem(orc.EULER2D, n, n, dx=1.0 / n, dy=1.0 / n)
    for _ in range(3):
        U, _ = orc.rk3_step(P, U)
        T, _ = orc.rk3_step(P, T)
    Tb = np.stack([T[0].T, T[2].T, T[1].T, T[3].T])
    assert np.abs(U - Tb).max() <= 1e-12 * np.abs(U).max()


def test_cfl_dt_definitions(orc):
    U = inputs.euler2d_ic(8, 6, seed=2)
    P = orc.problem(orc.EULER2D, 8, 6, dx=1 / 8, dy=1 / 6)
    rho, mu, mv, E = U
    u, v = mu / rho, mv / rho
    p = (GAMMA - 1) * (E - 0.5 * rho * (u * u + v * v))
    c = np.sqrt(GAMMA * p / rho)
    ax, ay = (np.abs(u) + c).max(), (np.abs(v) + c).max()
    assert orc.max_wavespeed(P, U, 0) == ax and orc.max_wavespeed(P, U, 1) == ay
    tx, ty = (1 / 8) / ax, (1 / 6) / ay
    assert orc.cfl_dt(P, U) == pytest.approx(0.5 * tx * ty / (tx + ty), rel=1e-15)


# ------------------------------------------------------------------ derivatives (adjoint reference)
@pytest.mark.parametrize("system,bc", [(1, 1), (1, 0), (2, 1), (0, 0)])
def test_oracle_jvp_matches_central_differences(orc, system, bc):
    """The forward-mode derivative of the discrete RHS against central differences of the
    oracle's own RHS on generic data (no flat fields, no ties)."""
    nx, ny = (30, 1) if system != 2 else (9, 8)
    U = inputs.random_smooth_state(system, nx, ny, seed=21)
    P = orc.problem(system, nx, ny, dx=0.1, dy=0.1, bc_x=bc, bc_y=bc)
    v = np.random.default_rng(4).normal(size=U.shape)
    _, dL = orc.rhs_jvp(P, U, v)
    h = 1e-6
    fd = (orc.rhs(P, U + h * v) - orc.rhs(P, U - h * v)) / (2 * h)
    assert np.abs(fd - dL).max() <= 1e-6 * np.abs(dL).max()
    _, dLq = orc.rhs_jvp_quad(P, U, v)
    assert np.abs(dLq - dL).max() <= 1e-10 * np.abs(dL).max()


def test_oracle_rollout_jvp_matches_central_differences(orc):
    n, steps = 128, 40
    U0 = inputs.adjoint_ic(n, seed=3)
    P = orc.problem(orc.EULER1D, n, 1, dx=10.0 / n, bc_x=orc.PERIODIC)
    dt = 0.5 * P.dx / orc.max_wavespeed(P, U0)
    v = np.random.default_rng(5).normal(size=U0.shape) * np.abs(U0)
    _, dU = orc.rollout_jvp(P, U0, v, dt, steps)
    h = 1e-7
    up, _ = orc.rollout_jvp(P, U0 + h * v, np.zeros_like(v), dt, steps)
    um, _ = orc.rollout_jvp(P, U0 - h * v, np.zeros_like(v), dt, steps)
    fd = (up - um) / (2 * h)
    assert np.abs(fd - dU).max() <= 1e-6 * np.abs(dU).max()


def test_rounding_flat_fields_make_the_exact_tangent_explode(orc):
    """Documented property of the scheme with eps = 1e-40: in the resting region of the
    Shu-Osher-type family the velocity is rounding noise after one step, the acoustic
    characteristic fields are flat to rounding and their weights are set by that noise, so
    the exact tangent of the discrete map grows by orders of magnitude per step."""
    n = 256
    U = inputs.euler1d_ic(n, seed=9)
    P = orc.problem(orc.EULER1D, n, 1, dx=10.0 / n, bc_x=orc.OUTFLOW)
    dt = 0.5 * P.dx / orc.max_wavespeed(P, U)
    v = np.random.default_rng(11).normal(size=U.shape) * np.abs(U)
    _, dU = orc.rollout_jvp(P, U, v, dt, 20)
    assert np.abs(dU).max() > 1e15
