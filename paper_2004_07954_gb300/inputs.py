"""Seeded synthetic initial conditions for the WENO-ZN solver.

This module only builds inputs: grids, primitive states drawn from seeded generators, and
their conversion to conserved variables with the ideal-gas energy relation of Sec. 4.3 /
Sec. 4.4 (E = p/(gamma-1) + rho |u|^2 / 2).  It holds none of the scheme's arithmetic and
both the CUDA path and the CPU oracle receive the arrays it returns.

Layout of every state: float64, planar, ``U[nvar][ny][nx]`` (x fastest), conserved
variables (rho, rho u[, rho v], E) or the scalar u.

Families (each a seeded generalisation of a paper set-up):
  * advection on [-1, 1], periodic, x_j = -1 + j dx: u0 = sin(pi x) and the first-order
    critical-point profile sin(pi x - sin(pi x)/pi);
  * 1D Euler on [-5, 5] with the Shu-Osher structure (Sec. 4.3.1): a constant left state for
    x < -4 and rho = 1 + A sin(k x), u = 0, p = 1 on the right; (rho, u, p)_L drawn from
    [1,4] x [0,3] x [1,11], A from [0.1, 0.3], k from [3, 8];
  * 2D Euler on [0, 1]^2, four-quadrant Riemann data split at (0.5, 0.5) (Sec. 4.4.1),
    per quadrant rho in [0.1, 1.5], u, v in [-1.2, 1.2], p in [0.03, 1.5];
  * smooth entropy waves (density sine carried by a constant velocity at constant pressure)
    whose exact solution is the translated profile;
  * the adjoint workload: a seeded smooth multi-wave state on the periodic domain [-5, 5]
    in which density, velocity and pressure all vary (no flat or resting region);
  * the four-wave advection profile of Sec. 4.2 (Gaussians, square, triangle, half ellipse)
    scaled by 1/A, and the two interacting blast waves of Sec. 4.3.2.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def cons_from_prim(rho, u, p, v=None, gamma=GAMMA) -> np.ndarray:
    """Conserved state from primitives; shape (3, ...) in 1D, (4, ...) in 2D."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), rho.shape)
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    if v is None:
        E = p / (gamma - 1.0) + 0.5 * rho * u * u
        return np.stack([rho, rho * u, E])
    v = np.broadcast_to(np.asarray(v, dtype=np.float64), rho.shape)
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return np.stack([rho, rho * u, rho * v, E])


# ---------------------------------------------------------------------------- advection
def advection_grid(n: int):
    dx = 2.0 / n
    return -1.0 + dx * np.arange(n), dx


def advection_profile(x, which: str):
    if which == "sin":
        return np.sin(np.pi * x)
    if which == "critical":
        return np.sin(np.pi * x - np.sin(np.pi * x) / np.pi)
    raise ValueError(which)


def advection_ic(n: int, which: str = "sin") -> np.ndarray:
    x, _ = advection_grid(n)
    return advection_profile(x, which).reshape(1, 1, n).copy()


def advection_exact(n: int, which: str, t: float, speed: float = 1.0) -> np.ndarray:
    x, _ = advection_grid(n)
    xs = np.mod(x - speed * t + 1.0, 2.0) - 1.0
    return advection_profile(xs, which).reshape(1, 1, n)


def advection_dt(n: int, T: float = 2.0):
    """Uniform step close to 0.1 dx^(5/3) that lands exactly on T: (dt, steps)."""
    dx = 2.0 / n
    steps = int(math.ceil(T / (0.1 * dx ** (5.0 / 3.0))))
    return T / steps, steps


# ---------------------------------------------------------------------------- 1D Euler
def euler1d_params(seed: int) -> dict:
    g = _rng(seed)
    rhoL, uL, pL = g.uniform(1.0, 4.0), g.uniform(0.0, 3.0), g.uniform(1.0, 11.0)
    amp, k = g.uniform(0.1, 0.3), g.uniform(3.0, 8.0)
    return {"rhoL": rhoL, "uL": uL, "pL": pL, "amp": amp, "k": k}


def euler1d_grid(n: int, a: float = -5.0, b: float = 5.0):
    dx = (b - a) / n
    return a + (np.arange(n) + 0.5) * dx, dx


def euler1d_ic(n: int, seed: int, x_s: float = -4.0) -> np.ndarray:
    prm = euler1d_params(seed)
    x, _ = euler1d_grid(n)
    left = x < x_s
    rho = np.where(left, prm["rhoL"], 1.0 + prm["amp"] * np.sin(prm["k"] * x))
    u = np.where(left, prm["uL"], 0.0)
    p = np.where(left, prm["pL"], 1.0)
    return cons_from_prim(rho, u, p).reshape(3, 1, n).copy()


def euler1d_batch(B: int, seed: int, n_min: int = 128, n_max: int = 16384):
    """Ragged batch of 1D Euler problems: sizes log-uniform in [n_min, n_max].

    Returns (sizes int64[B], offsets int64[B+1], U planar float64[3, sum(sizes)]) where
    instance b occupies columns offsets[b]:offsets[b+1] and uses seed `seed * 100003 + b`.
    """
    g = _rng(seed)
    sizes = np.round(np.exp(g.uniform(math.log(n_min), math.log(n_max), size=B))).astype(np.int64)
    offsets = np.zeros(B + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    U = np.empty((3, int(offsets[-1])), dtype=np.float64)
    for b in range(B):
        U[:, offsets[b]:offsets[b + 1]] = euler1d_ic(int(sizes[b]), seed * 100003 + b)[:, 0, :]
    return sizes, offsets, U


# ---------------------------------------------------------------------------- 2D Euler
def euler2d_params(seed: int) -> np.ndarray:
    """Quadrant states, rows: (x<=.5,y<=.5), (x<=.5,y>.5), (x>.5,y<=.5), (x>.5,y>.5);
    columns rho, u, v, p."""
    g = _rng(seed)
    q = np.empty((4, 4))
    for r in range(4):
        q[r] = [g.uniform(0.1, 1.5), g.uniform(-1.2, 1.2), g.uniform(-1.2, 1.2), g.uniform(0.03, 1.5)]
    return q


def euler2d_grid(nx: int, ny: int):
    dx, dy = 1.0 / nx, 1.0 / ny
    return (np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy, dx, dy


def euler2d_ic(nx: int, ny: int, seed: int) -> np.ndarray:
    q = euler2d_params(seed)
    x, y, _, _ = euler2d_grid(nx, ny)
    X, Y = np.meshgrid(x, y)          # shape (ny, nx)
    quad = np.where(X <= 0.5, np.where(Y <= 0.5, 0, 1), np.where(Y <= 0.5, 2, 3))
    rho, u, v, p = (q[quad, c] for c in range(4))
    return np.ascontiguousarray(cons_from_prim(rho, u, p, v))


# ---------------------------------------------------------------------------- entropy waves
def entropy_wave_1d(n: int, t: float = 0.0, u: float = 1.0, amp: float = 0.2):
    """Periodic [-1, 1], cell centres x_j = -1 + (j + 1/2) dx."""
    dx = 2.0 / n
    x = -1.0 + (np.arange(n) + 0.5) * dx
    rho = 1.0 + amp * np.sin(np.pi * (x - u * t))
    return cons_from_prim(rho, u, 1.0).reshape(3, 1, n).copy(), dx


def entropy_wave_2d(nx: int, ny: int, t: float = 0.0, u: float = 1.0, v: float = 0.5, amp: float = 0.2):
    """Periodic [-1, 1]^2, density sin(pi (x + y)) carried by (u, v)."""
    dx, dy = 2.0 / nx, 2.0 / ny
    x = -1.0 + (np.arange(nx) + 0.5) * dx
    y = -1.0 + (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    rho = 1.0 + amp * np.sin(np.pi * ((X - u * t) + (Y - v * t)))
    return np.ascontiguousarray(cons_from_prim(rho, u, 1.0, v)), dx, dy


def adjoint_params(seed: int) -> dict:
    g = _rng(seed)
    # whole waves on the period 10; the first one spans it once, so the state has no
    # shorter period (no exactly repeated maximum of |u| + c)
    m = np.concatenate([[1], g.integers(1, 4, size=3)])
    return {"A": g.uniform(0.1, 0.2), "B": g.uniform(0.05, 0.2), "C": g.uniform(0.05, 0.2),
            "u0": g.uniform(-0.5, 0.5), "k": 2.0 * np.pi * m / 10.0, "phi": g.uniform(0.0, 2.0 * np.pi, size=4)}


def adjoint_ic(n: int, seed: int) -> np.ndarray:
    """Smooth periodic 1D Euler state on [-5, 5] (cell centres): rho = 1 + A sin(k1 x + p1)
    + A/2 sin(k2 x + p2), u = u0 + B sin(k3 x + p3), p = 1 + C sin(k4 x + p4)."""
    q = adjoint_params(seed)
    x, _ = euler1d_grid(n)
    k, ph = q["k"], q["phi"]
    rho = 1.0 + q["A"] * np.sin(k[0] * x + ph[0]) + 0.5 * q["A"] * np.sin(k[1] * x + ph[1])
    u = q["u0"] + q["B"] * np.sin(k[2] * x + ph[2])
    p = 1.0 + q["C"] * np.sin(k[3] * x + ph[3])
    return cons_from_prim(rho, u, p).reshape(3, 1, n).copy()


def four_wave_profile(x, A: float = 1.0):
    """Sec. 4.2, case 1: on [-1, 1], (1/A) times a smooth combination of Gaussians on
    [-0.8, -0.6], a square wave on [-0.4, -0.2], a triangle on [0, 0.2] and a half ellipse on
    [0.4, 0.6], zero elsewhere; a = 0.5, z = -0.7, delta = 0.005, alpha = 10,
    beta = log 2 / (36 delta^2).  The ellipse term is centred at a -+ delta (the printed
    F(x, alpha, alpha -+ delta) reads a for alpha, as the centre a of the other term shows)."""
    x = np.asarray(x, dtype=np.float64)
    a, z, delta, alpha = 0.5, -0.7, 0.005, 10.0
    beta = math.log(2.0) / (36.0 * delta * delta)
    G = lambda zz: np.exp(-beta * (x - zz) ** 2)
    F = lambda aa: np.sqrt(np.maximum(1.0 - alpha * alpha * (x - aa) ** 2, 0.0))
    u = np.zeros_like(x)
    m = (x >= -0.8) & (x <= -0.6)
    u = np.where(m, (G(z - delta) + G(z + delta) + 4.0 * G(z)) / 6.0, u)
    u = np.where((x >= -0.4) & (x <= -0.2), 1.0, u)
    u = np.where((x >= 0.0) & (x <= 0.2), 1.0 - np.abs(10.0 * (x - 0.1)), u)
    m = (x >= 0.4) & (x <= 0.6)
    u = np.where(m, (F(a - delta) + F(a + delta) + 4.0 * F(a)) / 6.0, u)
    return u / A


def four_wave_ic(n: int, A: float = 1.0) -> np.ndarray:
    """The four-wave profile on the periodic advection grid x_j = -1 + j dx, dx = 2/n."""
    x, _ = advection_grid(n)
    return four_wave_profile(x, A).reshape(1, 1, n).copy()


def blast_wave_ic(n: int) -> np.ndarray:
    """Sec. 4.3.2, two interacting blast waves on [0, 1] (cell centres): rho = 1, u = 0,
    p = 1000 for x < 0.1, 0.01 for 0.1 <= x < 0.9, 100 for x >= 0.9."""
    x = (np.arange(n) + 0.5) / n
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    return cons_from_prim(np.ones(n), 0.0, p).reshape(3, 1, n).copy()


def random_smooth_state(system: int, nx: int, ny: int, seed: int) -> np.ndarray:
    """Positive, smooth-ish random Euler state (or scalar) for invariance tests."""
    g = _rng(seed)
    if system == 0:
        return g.uniform(-1.0, 1.0, size=(1, ny, nx))
    rho = g.uniform(0.5, 2.0, size=(ny, nx))
    u = g.uniform(-1.0, 1.0, size=(ny, nx))
    p = g.uniform(0.5, 2.0, size=(ny, nx))
    if system == 1:
        return cons_from_prim(rho, u, p)
    v = g.uniform(-1.0, 1.0, size=(ny, nx))
    return cons_from_prim(rho, u, p, v)
