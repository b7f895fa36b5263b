"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Tolerances: relative L-infinity <= 1e-12 for one RHS evaluation or one RK3 step and
<= 1e-9 at a final time (the targets stated for this solver); LF speeds and CFL steps are
compared bit for bit (a maximum is exact and both sides evaluate the per-cell speed in the
same IEEE operation order).
"""
import numpy as np
import pytest
import torch

from paper_2004_07954_gb300 import inputs

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12
FINAL_TOL = 1e-9


@pytest.fixture(scope="module")
def wz():
    from paper_2004_07954_gb300 import build, wenozn
    build.build()
    assert torch.cuda.is_available(), "CUDA device required"
    return wenozn


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_linf(got, want):
    scale = np.abs(want).max()
    return np.abs(got - want).max() / (scale if scale > 0 else 1.0)


def gpu_problem(wz, system, nx, ny=1, dx=0.1, dy=0.1, bc=1, bcy=None):
    return wz.wenozn_problem_init(system, nx, ny, dx, dy, bc_x=bc, bc_y=bc if bcy is None else bcy)


def orc_problem(orc, p):
    return orc.problem(p.system, p.nx, p.ny, dx=p.dx, dy=p.dy, bc_x=p.bc_x, bc_y=p.bc_y,
                       gamma=p.gamma, eps=p.eps, A=p.A, cfl=p.cfl, adv_speed=p.adv_speed)


# ------------------------------------------------------------------ reconstruction
@pytest.mark.parametrize("n", [1, 2, 5, 64, 255, 256, 300, 1000, 4099])
@pytest.mark.parametrize("side", [1, -1])
def test_reconstruct_random(wz, orc, n, side):
    g = np.random.default_rng(n * 7 + side)
    for scale in (1.0, 1e-3, 1e4):
        f = g.normal(size=n + 6) * scale
        f[g.random(n + 6) < 0.1] += 5 * scale         # sprinkle jumps
        out = torch.empty(n + 1, dtype=torch.float64, device="cuda")
        wz.wenozn_reconstruct(dev(f), out, side)
        want = orc.reconstruct(f, side)
        assert np.abs(host(out) - want).max() <= STEP_TOL * np.abs(f).max()


def test_reconstruct_polynomial_and_step(wz, orc):
    x = np.arange(-3, 40, dtype=np.float64)
    for f in (2.0 + 0 * x, 1.0 - 2 * x + 3 * x * x + 0.5 * x ** 3, np.where(x < 11, 0.0, 1.0)):
        out = torch.empty(f.size - 5, dtype=torch.float64, device="cuda")
        wz.wenozn_reconstruct(dev(f), out, 1)
        want = orc.reconstruct(f, 1)
        assert np.abs(host(out) - want).max() <= STEP_TOL * np.abs(f).max()


def test_table3_critical_points_on_gpu(wz, orc):
    """The FP64-resolvable rows of the paper's critical-point table, through the CUDA
    reconstruction (f^+_{1/2} - f^+_{-1/2}) / dx against f'(0)."""
    from conftest import read_golden
    rows = {1: range(0, 2), 2: range(0, 5), 3: range(0, 8)}
    for k, j, _z, _za, zn in read_golden("table3_critical_point.txt"):
        k, j = int(k), int(j)
        if j not in rows[k]:
            continue
        dx = 0.025 / 2 ** j
        xs = dx * np.arange(-3, 4)
        f = xs ** k * np.exp(xs)
        out = torch.empty(2, dtype=torch.float64, device="cuda")
        wz.wenozn_reconstruct(dev(f), out, 1)
        fh = host(out)
        err = abs((fh[1] - fh[0]) / dx - (1.0 if k == 1 else 0.0))
        assert err == pytest.approx(zn, rel=1e-4)


def test_newton_reciprocal_within_one_ulp(wz):
    """The reciprocal behind f^ = num/den (Newton-Raphson on the hardware approximation)
    stays within one ulp of CUDA's IEEE 1/d over the whole normal range it is used on."""
    g = np.random.default_rng(7)
    d = np.ldexp(g.uniform(1.0, 2.0, 200000), g.integers(-1000, 1000, 200000))
    d = np.concatenate([d, [1.0, 2.0, 3.0, 1e-300, 1e300, 0.1, 7.0, np.nextafter(2.0, 0)]])
    fast, ieee = wz.wenozn_check_reciprocal(dev(d))
    f, i = host(fast), host(ieee)
    assert np.array_equal(i, 1.0 / d)                     # CUDA's division is IEEE
    ulp = np.spacing(np.abs(i))
    assert np.all(np.abs(f - i) <= ulp)


def test_fp64_fma_rate(wz):
    """The FP64 FMA probe reports a rate between half and all of the nominal peak
    (2 FMA lanes per SM per clock, 152 SMs, 2070 MHz) and rejects bad arguments."""
    g = wz.wenozn_fp64_fma_rate(1 << 15)
    assert 0.5 * 1258.6 < g < 1.02 * 1258.6
    for bad in (0, 3, (1 << 32) + 1):
        with pytest.raises(wz.WenoznError):
            wz.wenozn_fp64_fma_rate(bad)


# ------------------------------------------------------------------ ghosts and LF speeds
@pytest.mark.parametrize("bc", [0, 1])
def test_fill_ghosts(wz, orc, bc):
    g = np.random.default_rng(bc)
    nx, ny = 9, 7
    p = gpu_problem(wz, 2, nx, ny, bc=bc)
    U = g.normal(size=(4, ny + 6, nx + 6))
    t = dev(U)
    wz.wenozn_fill_ghosts(p, t)
    want = U.copy()
    for k in range(4):
        for r in range(3, ny + 3):
            want[k, r] = orc.fill_ghosts_line(want[k, r], bc)
        for c in range(nx + 6):
            want[k, :, c] = orc.fill_ghosts_line(want[k, :, c].copy(), bc)
    assert np.array_equal(host(t), want)
    p1 = gpu_problem(wz, 1, nx, bc=bc)
    U1 = g.normal(size=(3, nx + 6))
    t1 = dev(U1)
    wz.wenozn_fill_ghosts(p1, t1)
    for k in range(3):
        assert np.array_equal(host(t1)[k], orc.fill_ghosts_line(U1[k], bc))


@pytest.mark.parametrize("system,nx,ny", [(1, 1000, 1), (2, 77, 53), (1, 1 << 20, 1)])
def test_max_wavespeed_bit_exact(wz, orc, system, nx, ny):
    if system == 1:
        U = inputs.euler1d_ic(nx, seed=5)
    else:
        U = inputs.euler2d_ic(nx, ny, seed=5)
    p = gpu_problem(wz, system, nx, ny)
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    wz.wenozn_max_wavespeed(p, dev(U), a)
    P = orc_problem(orc, p)
    got = host(a)
    assert got[0] == orc.max_wavespeed(P, U, 0)
    if system == 2:
        assert got[1] == orc.max_wavespeed(P, U, 1)


# ------------------------------------------------------------------ RHS
RHS_CASES = [
    (0, 1, 1, 0), (0, 37, 1, 0), (0, 700, 1, 0), (0, 1031, 1, 1),
    (1, 1, 1, 1), (1, 5, 1, 0), (1, 200, 1, 1), (1, 513, 1, 1), (1, 1100, 1, 0),
    (2, 1, 1, 1), (2, 5, 3, 0), (2, 37, 21, 1), (2, 150, 45, 1), (2, 70, 130, 0), (2, 64, 64, 1),
]


def _rand_state(system, nx, ny, seed):
    if system == 0:
        return inputs.random_smooth_state(0, nx, ny, seed)
    if system == 1:
        return inputs.euler1d_ic(nx, seed) if nx >= 20 else inputs.random_smooth_state(1, nx, ny, seed)
    if nx >= 8 and ny >= 8:
        return inputs.euler2d_ic(nx, ny, seed)
    return inputs.random_smooth_state(2, nx, ny, seed)


@pytest.mark.parametrize("system,nx,ny,bc", RHS_CASES)
def test_rhs_parity(wz, orc, system, nx, ny, bc):
    U = _rand_state(system, nx, ny, seed=nx + ny)
    p = gpu_problem(wz, system, nx, ny, dx=1.0 / nx, dy=1.0 / ny, bc=bc)
    S = wz.Solver(p)
    L = host(S.rhs(dev(U)))
    want = orc.rhs(orc_problem(orc, p), U)
    assert rel_linf(L, want) <= STEP_TOL
    assert S.status() == 0


@pytest.mark.parametrize("nx,ny,bc", [(37, 21, 1), (70, 130, 0), (129, 64, 1), (256, 33, 0)])
def test_flux_sweeps_and_both_in_one_launch(wz, orc, nx, ny, bc):
    """wenozn_flux: the x sweep, the y sweep and both in one launch (the form the RHS and the
    RK3 steps run) give the same interface fluxes bit for bit, and their differences are the
    oracle's right-hand side."""
    U = _rand_state(2, nx, ny, seed=nx + 2 * ny)
    p = gpu_problem(wz, 2, nx, ny, dx=1.0 / nx, dy=1.0 / ny, bc=bc)
    t = dev(U)
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    wz.wenozn_max_wavespeed(p, t, a)
    out = [torch.empty(wz.flux_shape(p, d), dtype=torch.float64, device="cuda") for d in (0, 1, 2)]
    for d in (0, 1, 2):
        wz.wenozn_flux(p, t, a, d, out[d])
    X, Y, both = (host(o) for o in out)
    assert np.array_equal(both[:X.size].reshape(X.shape), X)
    assert np.array_equal(both[X.size:].reshape(Y.shape), Y)
    L = -(X[:, :, 1:] - X[:, :, :-1]) * nx - (Y[:, 1:, :] - Y[:, :-1, :]) * ny
    assert rel_linf(L, orc.rhs(orc_problem(orc, p), U)) <= STEP_TOL
    with pytest.raises(wz.WenoznError):
        p1 = gpu_problem(wz, 1, nx)
        wz.wenozn_flux(p1, dev(_rand_state(1, nx, 1, seed=1)), a, 2, out[2])


# ------------------------------------------------------------------ one RK3 step
@pytest.mark.parametrize("system,nx,ny,bc", RHS_CASES)
def test_rk3_step_parity(wz, orc, system, nx, ny, bc):
    U = _rand_state(system, nx, ny, seed=nx * 3 + ny)
    p = gpu_problem(wz, system, nx, ny, dx=1.0 / nx, dy=1.0 / ny, bc=bc)
    S = wz.Solver(p)
    t = dev(U)
    dt = S.step(t, return_dt=True)
    want, dt_o = orc.rk3_step(orc_problem(orc, p), U)
    assert dt == dt_o
    assert rel_linf(host(t), want) <= STEP_TOL


@pytest.mark.parametrize("system,nx,ny,split", [(2, 70, 53, 0), (1, 777, 1, 0), (0, 300, 1, 0), (2, 40, 33, 1),
                                                 (1, 500, 1, 1)])
def test_rk3_run_equals_repeated_steps(wz, system, nx, ny, split):
    """The chained steps (LF speeds of each new state from the last stage, rotating slots)
    give the results of single steps bit for bit, with CFL and with fixed steps."""
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / max(ny, 1), split=split)
    U0 = (inputs.euler2d_ic(nx, ny, 2) if system == 2 else
          inputs.euler1d_ic(nx, 2) if system == 1 else inputs.advection_ic(nx, "sin"))
    for dt in (0.0, 1e-4):
        S = wz.Solver(p)
        a, b = dev(U0), dev(U0)
        for _ in range(7):
            S.step(a, dt=dt)
        S.steps(b, 7, dt=dt)
        assert torch.equal(a, b)
        assert S.status() == 0


@pytest.mark.parametrize("bc", [0, 1, 2])
def test_large_1d_step_parity(wz, orc, bc):
    """A 1D grid on the large-grid kernels (512-interface flux tiles, 256-thread update
    blocks): one step against the oracle for every boundary, with a ragged last tile, CFL,
    clipped and fixed steps, and the chained run equal to repeated steps."""
    n = 200_000                                      # 390 full flux tiles + 321 interfaces
    U0 = inputs.euler1d_ic(n, seed=9)
    if bc == 2:
        U0 = U0.copy()
        U0[1] *= 0.0                                 # at rest next to the walls
    p = gpu_problem(wz, 1, n, dx=10.0 / n, bc=bc)
    P = orc_problem(orc, p)
    for dt, trem in ((0.0, 0.0), (0.0, 1e-6), (2e-5, 0.0)):
        S = wz.Solver(p)
        t = dev(U0)
        got = S.step(t, dt=dt, t_remaining=trem, return_dt=True)
        want, used = orc.rk3_step(P, U0, dt, trem)
        assert got == used
        assert rel_linf(host(t), want) <= STEP_TOL
        assert S.status() == 0
    S = wz.Solver(p)
    a, b = dev(U0), dev(U0)
    for _ in range(3):
        S.step(a)
    S.steps(b, 3)
    assert torch.equal(a, b)


def test_2d_chained_steps_repeatable_at_the_benchmark_size(wz):
    """4096^2, six chained steps (programmatically dependent launches), three times:
    bit-identical states and steps."""
    n = 4096
    p = gpu_problem(wz, 2, n, n, dx=1.0 / n, dy=1.0 / n)
    U0 = dev(inputs.euler2d_ic(n, n, seed=0))
    S = wz.Solver(p)
    ref, dts = None, None
    for _ in range(3):
        U = U0.clone()
        S.steps(U, 6)
        dt = wz.wenozn_workspace_dt(S.ws).item()
        if ref is None:
            ref, dts = U, dt
        else:
            assert torch.equal(U, ref) and dt == dts
    assert S.status() == 0


@pytest.mark.parametrize("system,nx,ny,split", [(0, 300, 1, 0), (1, 1000, 1, 0), (1, 700, 1, 1), (2, 77, 53, 0),
                                                 (2, 40, 33, 1)])
def test_cfl_dt_bit_exact(wz, orc, system, nx, ny, split):
    """wenozn_cfl_dt equals the oracle's CFL step (Sec. 4.3 / 4.4) and the step the RK3 call
    takes, bit for bit."""
    U = (inputs.advection_ic(nx, "sin") if system == 0 else
         inputs.euler1d_ic(nx, 6) if system == 1 else inputs.euler2d_ic(nx, ny, 6))
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / ny, split=split)
    S = wz.Solver(p)
    dt = wz.wenozn_cfl_dt(p, dev(U), S.ws)
    assert dt == orc.cfl_dt(orc_problem(orc, p), U)
    assert dt == S.step(dev(U), return_dt=True)
    assert S.status() == 0


@pytest.mark.parametrize("system,nx,ny", [(1, 5000, 1), (2, 200, 150)])
def test_rk3_step_host_equals_device_step(wz, system, nx, ny):
    """The host-buffer step (copy in, step, copy out in one call) gives the device step's
    state and time step bit for bit: pinned and pageable buffers, separate and shared in/out
    buffers, CFL, fixed and clipped steps, three steps chained through host memory."""
    U0 = inputs.euler1d_ic(nx, 3) if system == 1 else inputs.euler2d_ic(nx, ny, 3)
    dx = 10.0 / nx if system == 1 else 1.0 / nx        # the families' domains: the fixed step is stable
    p = wz.wenozn_problem_init(system, nx, ny, dx, 1.0 / ny)
    A, B = wz.Solver(p), wz.Solver(p)
    U_dev = torch.empty(p.shape, dtype=torch.float64, device="cuda")
    for dt, trem in ((0.0, 0.0), (1e-4, 0.0), (0.0, 1e-5)):
        for pinned in (True, False):
            a = dev(U0)
            want_dt = A.step(a, dt=dt, t_remaining=trem, return_dt=True)
            h_in = torch.from_numpy(U0.copy())
            h_out = torch.empty_like(h_in)
            if pinned:
                h_in, h_out = h_in.pin_memory(), h_out.pin_memory()
            got_dt = wz.wenozn_rk3_step_host(p, h_in, h_out, U_dev, B.ws, dt, trem, return_dt=True)
            assert got_dt == want_dt
            assert torch.equal(h_out, a.cpu())
    a = dev(U0)
    h = torch.from_numpy(U0.copy()).pin_memory()
    for _ in range(3):
        A.step(a)
        wz.wenozn_rk3_step_host(p, h, h, U_dev, B.ws)
    torch.cuda.synchronize()
    assert torch.equal(h, a.cpu())
    assert A.status() == 0 and B.status() == 0


@pytest.mark.parametrize("copy_streams,count", [(True, 5), (False, 5), (True, 1), (True, 2), (False, 1)])
def test_rk3_stream_host_equals_device_steps(wz, copy_streams, count):
    """The streaming host-buffer call gives, for each of its states, the device step's result
    bit for bit: `count` different states (CFL and fixed steps; one and two states never reuse
    a staging buffer), outputs distinct or equal to the inputs, with and without separate copy
    streams, and the call ordered on its stream."""
    nx, ny = 160, 120
    p = wz.wenozn_problem_init(2, nx, ny, 1.0 / nx, 1.0 / ny)
    states = [inputs.euler2d_ic(nx, ny, 20 + k) for k in range(count)]
    A, B = wz.Solver(p), wz.Solver(p)
    for dt in (0.0, 2e-4):
        want = []
        for U0 in states:
            a = dev(U0)
            A.step(a, dt=dt)
            want.append(a.cpu())
        ins = [torch.from_numpy(U0.copy()).pin_memory() for U0 in states]
        outs = [torch.empty_like(x).pin_memory() for x in ins[:3]] + ins[3:]     # beyond three: in place
        if count <= 2:
            outs[-1] = ins[-1]
        d0, d1 = (torch.empty(p.shape, dtype=torch.float64, device="cuda") for _ in range(2))
        kw = {"upload_stream": torch.cuda.Stream(), "download_stream": torch.cuda.Stream()} if copy_streams else {}
        wz.wenozn_rk3_stream_host(p, ins, outs, d0, d1, B.ws, dt, **kw)
        torch.cuda.current_stream().synchronize()          # the call is ordered on its stream
        for k in range(count):
            assert torch.equal(outs[k], want[k]), (dt, k)
    assert A.status() == 0 and B.status() == 0


def test_rk3_fixed_and_clipped_dt(wz, orc):
    n = 300
    U = inputs.euler1d_ic(n, seed=2)
    p = gpu_problem(wz, 1, n, dx=10.0 / n)
    S = wz.Solver(p)
    P = orc_problem(orc, p)
    for dt, trem in ((1e-3, 0.0), (0.0, 1e-4), (5e-3, 2e-3)):
        t = dev(U)
        got = S.step(t, dt=dt, t_remaining=trem, return_dt=True)
        want, used = orc.rk3_step(P, U, dt, trem)
        assert got == used
        assert rel_linf(host(t), want) <= STEP_TOL


# ------------------------------------------------------------------ final time
# (advection orders, 1D Euler to t = 1.8, 2D Euler over 200 steps and batched instances to
# their final time, all under one parity rule: tests/test_gpu_final_time.py)


# ------------------------------------------------------------------ full sizes
@pytest.mark.parametrize("system,n_big,n_tile", [(2, 4096, 64), (1, 1 << 20, 256)])
def test_full_size_tiled_periodic(wz, orc, system, n_big, n_tile):
    """At the benchmark's sizes (4096^2 2D, 2^20 1D) and launch configuration: a periodic
    grid tiled with copies of a small periodic problem evolves exactly like the small
    problem (same global LF speeds, same stencils), so every sampled cell of one RK3 step
    compares against the oracle run on the small grid."""
    reps = n_big // n_tile
    if system == 2:
        small = inputs.euler2d_ic(n_tile, n_tile, seed=3)
        big = np.tile(small, (1, reps, reps))
        p = gpu_problem(wz, 2, n_big, n_big, dx=1.0 / n_big, dy=1.0 / n_big, bc=0)
        ps = orc.problem(2, n_tile, n_tile, dx=1.0 / n_big, dy=1.0 / n_big, bc_x=0, bc_y=0)
    else:
        small = inputs.euler1d_ic(n_tile, seed=3)
        big = np.tile(small, (1, 1, reps))
        p = gpu_problem(wz, 1, n_big, dx=1.0 / n_big, bc=0)
        ps = orc.problem(1, n_tile, 1, dx=1.0 / n_big, bc_x=0)
    S = wz.Solver(p)
    t = dev(big)
    del big
    dt = S.step(t, return_dt=True)
    want, dt_o = orc.rk3_step(ps, small)
    assert dt == dt_o
    got = host(t)
    g = np.random.default_rng(0)
    if system == 2:
        js, is_ = g.integers(0, n_big, 4096), g.integers(0, n_big, 4096)
        a = got[:, js, is_]
        b = want[:, js % n_tile, is_ % n_tile]
        # and whole tiles at the corners and the centre
        for (r, c) in ((0, 0), (reps - 1, reps - 1), (reps // 2, reps // 3)):
            blk = got[:, r * n_tile:(r + 1) * n_tile, c * n_tile:(c + 1) * n_tile]
            assert rel_linf(blk, want) <= STEP_TOL
    else:
        is_ = g.integers(0, n_big, 65536)
        a = got[:, 0, is_]
        b = want[:, 0, is_ % n_tile]
    assert np.abs(a - b).max() <= STEP_TOL * np.abs(want).max()
    assert S.status() == 0


def test_benchmark_workload_full_grid(wz, orc):
    """The benchmark's own workload (2D Euler 4096^2, the seeded four-quadrant problem with
    seed 0, outflow), through the chained call the benchmark times: every cell of one RK3 step
    against the oracle's step of the same data, the CFL step bit for bit; and the CFL step of
    a two-step chain's second step, which comes from the update kernel's screened LF speeds,
    against the oracle's for the GPU's state after the first step."""
    n = 4096
    U0 = inputs.euler2d_ic(n, n, seed=0)
    p = gpu_problem(wz, 2, n, n, dx=1.0 / n, dy=1.0 / n, bc=1)
    P = orc_problem(orc, p)
    one, two = wz.Solver(p), wz.Solver(p)
    t1, t2 = dev(U0), dev(U0)
    one.steps(t1, 1)
    two.steps(t2, 2)
    torch.cuda.synchronize()
    dt1 = wz.wenozn_workspace_dt(one.ws).item()
    dt2 = wz.wenozn_workspace_dt(two.ws).item()
    assert one.status() == 0 and two.status() == 0
    del t2, two
    want, dt_o = orc.rk3_step(P, U0)
    del U0
    assert dt1 == dt_o
    got = host(t1)
    assert rel_linf(got, want) <= STEP_TOL
    del want
    assert dt2 == orc.cfl_dt(P, got)


# ------------------------------------------------------------------ invariants on the GPU
def test_conservation_periodic_gpu(wz):
    n = 256
    U0 = inputs.euler2d_ic(n, n, seed=4)
    p = gpu_problem(wz, 2, n, n, dx=1.0 / n, dy=1.0 / n, bc=0)
    S = wz.Solver(p)
    t = dev(U0)
    for _ in range(5):
        S.step(t)
    got = host(t)
    for k in range(4):
        assert abs(got[k].sum() - U0[k].sum()) <= 1e-12 * np.abs(U0[k]).sum()


def test_free_stream_gpu(wz):
    p = gpu_problem(wz, 2, 100, 70, bc=1)
    prim = inputs.cons_from_prim(np.array(1.3), 0.7, 2.1, -0.4)
    U = np.broadcast_to(prim.reshape(4, 1, 1), (4, 70, 100)).copy()
    L = host(wz.Solver(p).rhs(dev(U)))
    assert np.abs(L).max() <= 1e-13


def test_nonfinite_status(wz):
    n = 64
    U = inputs.euler1d_ic(n, seed=0)
    U[0, 0, 10] = np.nan
    p = gpu_problem(wz, 1, n, dx=0.1)
    S = wz.Solver(p)
    S.step(dev(U), dt=1e-4)
    assert S.status(clear=True) & (1 << wz.WENOZN_ENONFINITE)
    assert S.status() == 0
    U[0, 0, 10] = -1.0
    S.step(dev(U), dt=1e-4)
    assert S.status() & (1 << wz.WENOZN_ENONFINITE)
    # the same bits through the per-stream query, which clears them
    assert wz.wenozn_last_error() & (1 << wz.WENOZN_ENONFINITE)
    assert wz.wenozn_last_error() == 0 and S.status() == 0
    S.step(dev(inputs.euler1d_ic(n, seed=0)), dt=1e-4)
    assert wz.wenozn_last_error() == 0


def test_invalid_arguments_gpu(wz):
    p = gpu_problem(wz, 1, 64)
    S = wz.Solver(p)
    small_ws = S.ws[:64]
    U = dev(inputs.euler1d_ic(64, 0))
    with pytest.raises(wz.WenoznError) as ei:
        wz.wenozn_rk3_step(p, U, small_ws)
    assert ei.value.code == wz.WENOZN_ENOMEM_WS
    with pytest.raises(wz.WenoznError):
        wz.wenozn_rhs(p, U, U, S.ws)
    with pytest.raises(ValueError):
        S.step(U.float())
