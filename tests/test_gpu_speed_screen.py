"""The screened LF-speed maximum against the oracle's exact maximum, bit for bit.

The kernels estimate |u_n| + c of every cell in single precision and evaluate the IEEE
speed only where the estimate comes within 2^-11 of the running maximum of the estimates,
or where the state lies outside the estimate's proven range (very fast flows, magnitudes
beyond 2^+-30); bit-identical states reuse the last exact speed.  These fields are built
to defeat a wrong screen: maxima that differ from their rivals by less than the estimate's
error, planted late in the grid-stride order, in states without an estimate, in constant
regions with one cell a few ulps faster, and tiny or signed-zero momenta.
"""
import numpy as np
import pytest
import torch

from paper_2004_07954_gb300 import inputs

pytestmark = pytest.mark.gpu

GAMMA = 1.4
NONFINITE_BIT = 1 << 4


@pytest.fixture(scope="module")
def wz():
    from paper_2004_07954_gb300 import build, wenozn
    build.build()
    assert torch.cuda.is_available(), "CUDA device required"
    return wenozn


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def orc_problem(orc, p):
    return orc.problem(p.system, p.nx, p.ny, dx=p.dx, dy=p.dy, bc_x=p.bc_x, bc_y=p.bc_y,
                       gamma=p.gamma, eps=p.eps, A=p.A, cfl=p.cfl, adv_speed=p.adv_speed)


def prim_state(system, rho, u, p, v=None):
    U = inputs.cons_from_prim(np.asarray(rho, float), np.asarray(u, float), np.asarray(p, float),
                              None if system == 1 else np.asarray(v, float))
    return U


def field(kind, system, nx, ny, seed):
    """[nvar][ny][nx] conserved state of the named adversarial family."""
    g = np.random.default_rng(seed)
    shape = (ny, nx)
    n = nx * ny
    c0 = np.sqrt(GAMMA)                          # sound speed of rho = p = 1
    rho = np.ones(shape)
    p = np.ones(shape)
    u = np.zeros(shape)
    v = np.zeros(shape)
    if kind == "near_tie":
        # every cell within 1e-6 of the same speed, far below the estimate's resolution
        u = 0.5 * (1.0 + g.uniform(-1e-6, 1e-6, size=shape))
        v = 0.3 * (1.0 + g.uniform(-1e-6, 1e-6, size=shape))
    elif kind == "near_tie_ulps":
        u = 0.5 * (1.0 + g.integers(-8, 9, size=shape) * 2.0 ** -52)
        v = 0.3 * (1.0 + g.integers(-8, 9, size=shape) * 2.0 ** -52)
    elif kind == "planted":
        # random field; 24 cells planted late in the order, rivals within 1e-6 of each other
        rho = g.uniform(0.5, 2.0, size=shape)
        p = g.uniform(0.5, 2.0, size=shape)
        u = g.uniform(-1.0, 1.0, size=shape)
        v = g.uniform(-1.0, 1.0, size=shape)
        flat = g.choice(np.arange(n // 2, n), size=24, replace=False)
        top = 4.0
        for k, f in enumerate(flat):
            j, i = divmod(int(f), nx)
            rho[j, i], p[j, i] = 1.0, 1.0
            u[j, i] = (top - c0) * (1.0 + 1e-7 * g.uniform(-1, 1)) * (-1 if k % 2 else 1)
            v[j, i] = (top - c0) * (1.0 + 1e-7 * g.uniform(-1, 1)) * (-1 if k % 3 else 1)
    elif kind == "constant_one_up":
        u = np.full(shape, 0.5)
        v = np.full(shape, 0.3)
        f = int(g.integers(n // 2, n))
        j, i = divmod(f, nx)
        u[j, i] = np.nextafter(np.nextafter(0.5, 1.0), 1.0)
        v[j, i] = np.nextafter(0.3, 1.0)
    elif kind == "hypersonic":
        # Mach ~ 10 cells carry no estimate; their maximum is the field's
        rho = g.uniform(0.5, 2.0, size=shape)
        p = g.uniform(0.5, 2.0, size=shape)
        u = g.uniform(-1.0, 1.0, size=shape)
        v = g.uniform(-1.0, 1.0, size=shape)
        sel = g.random(shape) < 0.01
        c = np.sqrt(GAMMA * p / rho)
        u[sel] = 10.0 * c[sel] * g.uniform(0.99, 1.0, size=sel.sum())
        v[sel] = -10.0 * c[sel] * g.uniform(0.99, 1.0, size=sel.sum())
    elif kind == "ranges":
        # densities and energies beyond 2^+-30 next to ordinary ones, similar speeds
        scale = g.choice([1e-12, 1.0, 1e12], size=shape)
        rho = scale * g.uniform(0.9, 1.1, size=shape)
        p = scale * g.uniform(0.9, 1.1, size=shape)
        u = g.uniform(-0.5, 0.5, size=shape)
        v = g.uniform(-0.5, 0.5, size=shape)
    elif kind == "tiny_momentum":
        rho = g.uniform(0.5, 2.0, size=shape)
        p = g.uniform(0.5, 2.0, size=shape)
        u = g.choice([0.0, -0.0, 1e-35, -1e-35, 1e-200, 3e-31, 5e-310, -5e-310], size=shape)
        v = g.choice([0.0, -0.0, 1e-36, -1e-300, 2e-31], size=shape)
    else:
        raise ValueError(kind)
    if system == 1:
        return prim_state(1, rho, u, p)
    return prim_state(2, rho, u, p, v)


KINDS = ["near_tie", "near_tie_ulps", "planted", "constant_one_up", "hypersonic", "ranges", "tiny_momentum"]
# (nx, ny): few cells (64-thread blocks), one batch per block, several batches per block
SIZES = {1: [(5000, 1), (200_000, 1), (1_000_003, 1)], 2: [(71, 70), (500, 400), (1000, 777)]}


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("system", [1, 2])
@pytest.mark.parametrize("size", [0, 1, 2])
def test_max_wavespeed_screen(wz, orc, kind, system, size):
    nx, ny = SIZES[system][size]
    U = field(kind, system, nx, ny, seed=100 * size + system)
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / ny)
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    wz.wenozn_max_wavespeed(p, dev(U), a, st)
    P = orc_problem(orc, p)
    got = a.cpu().numpy()
    assert int(st.item()) == 0
    assert got[0] == orc.max_wavespeed(P, U, 0)
    if system == 2:
        assert got[1] == orc.max_wavespeed(P, U, 1)


@pytest.mark.parametrize("gamma", [1.1, 5.0 / 3.0, 3.0])
@pytest.mark.parametrize("system", [1, 2])
def test_screen_other_gammas(wz, orc, gamma, system):
    """The estimate's bound does not depend on gamma (gamma (gamma - 1) enters rounded once)."""
    nx, ny = (400_000, 1) if system == 1 else (640, 600)
    U = field("near_tie", system, nx, ny, seed=21)
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / ny)
    p.gamma = gamma
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    wz.wenozn_max_wavespeed(p, dev(U), a, st)
    P = orc_problem(orc, p)
    got = a.cpu().numpy()
    assert int(st.item()) == 0
    assert got[0] == orc.max_wavespeed(P, U, 0)
    if system == 2:
        assert got[1] == orc.max_wavespeed(P, U, 1)


@pytest.mark.parametrize("system", [1, 2])
@pytest.mark.parametrize("bad", ["negative_pressure", "nan"])
def test_screen_keeps_status(wz, orc, system, bad):
    nx, ny = (600_000, 1) if system == 1 else (800, 700)
    U = field("planted", system, nx, ny, seed=7)
    g = np.random.default_rng(11)
    f = int(g.integers(nx * ny // 2, nx * ny))
    j, i = divmod(f, nx)
    if bad == "nan":
        U[0, j, i] = np.nan
    else:
        U[-1, j, i] = 0.25 * U[1, j, i] ** 2 / U[0, j, i]      # E below the kinetic energy
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / ny)
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    wz.wenozn_max_wavespeed(p, dev(U), a, st)
    assert int(st.item()) & NONFINITE_BIT


def stage_alphas(wz, p, ws):
    U1, U2, A = wz.workspace_stages(p, ws)
    off = A.data_ptr() - ws.data_ptr()
    raw = ws[off:off + 48].view(torch.float64).cpu().numpy().reshape(3, 2)
    return U1.cpu().numpy(), U2.cpu().numpy(), raw


STEP_CASES = [
    ("four_quadrant", 2, 700, 500), ("four_quadrant", 2, 97, 61), ("planted", 2, 640, 600),
    ("shu_osher", 1, 1 << 20, 1), ("shu_osher", 1, 3001, 1), ("near_tie", 1, 400_000, 1),
]


@pytest.mark.parametrize("kind,system,nx,ny", STEP_CASES)
def test_stage_speeds_screen(wz, orc, kind, system, nx, ny):
    """The update kernel's screened speeds of the stage states U^(1), U^(2) are the exact
    maxima over those (GPU-computed) states."""
    if kind == "four_quadrant":
        U = inputs.euler2d_ic(nx, ny, seed=3)
    elif kind == "shu_osher":
        U = inputs.euler1d_ic(nx, seed=3)
    else:
        U = field(kind, system, nx, ny, seed=5)
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / ny)
    S = wz.Solver(p)
    t = dev(U)
    S.step(t)
    torch.cuda.synchronize()
    assert S.status() == 0
    U1, U2, raw = stage_alphas(wz, p, S.ws)
    P = orc_problem(orc, p)
    for s, Us in ((1, U1), (2, U2)):
        assert raw[s, 0] == orc.max_wavespeed(P, Us, 0), f"stage {s} x"
        if system == 2:
            assert raw[s, 1] == orc.max_wavespeed(P, Us, 1), f"stage {s} y"


FIELD_CASES = [("four_quadrant", 2, 700, 500), ("planted", 2, 640, 600), ("near_tie", 2, 500, 400),
               ("shu_osher", 1, 1 << 20, 1), ("near_tie", 1, 400_000, 1), ("tiny_momentum", 1, 300_000, 1),
               ("constant_one_up", 2, 600, 600)]


@pytest.mark.parametrize("kind,system,nx,ny", FIELD_CASES)
def test_stage_field_speeds_screen(wz, orc, kind, system, nx, ny):
    """Per-field LF splitting: the update kernel's screened per-field maxima |u-c|, |u|, |u+c|
    (and with v) of U^(1), U^(2) are the exact maxima over those states."""
    if kind == "four_quadrant":
        U = inputs.euler2d_ic(nx, ny, seed=6)
    elif kind == "shu_osher":
        U = inputs.euler1d_ic(nx, seed=6)
    else:
        U = field(kind, system, nx, ny, seed=8)
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / ny)
    p.split = wz.WENOZN_SPLIT_LF_FIELD
    S = wz.Solver(p)
    t = dev(U)
    S.step(t)
    torch.cuda.synchronize()
    assert S.status() == 0
    U1, U2, A = wz.workspace_stages(p, S.ws)
    off = A.data_ptr() - S.ws.data_ptr()
    raw = S.ws[off:off + 48 + 144].view(torch.float64).cpu().numpy()
    af = raw[6:].reshape(3, 2, 3)
    P = orc_problem(orc, p)
    P.split = p.split
    for slot, Us in ((1, U1.cpu().numpy()), (2, U2.cpu().numpy())):
        assert raw[2 * slot] == orc.max_wavespeed(P, Us, 0)
        for d in range(2 if system == 2 else 1):
            for k in range(3):
                assert af[slot, d, k] == orc.field_speed(P, Us, d, k), (slot, d, k)


@pytest.mark.parametrize("system,nx,ny", [(2, 700, 500), (1, 1 << 20, 1)])
def test_chained_step_dt_screen(wz, orc, system, nx, ny):
    """In a chained run the last stage's screened speeds give the next step's CFL dt."""
    U = inputs.euler2d_ic(nx, ny, seed=4) if system == 2 else inputs.euler1d_ic(nx, seed=4)
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / ny)
    one, two = wz.Solver(p), wz.Solver(p)
    a, b = dev(U), dev(U)
    one.steps(a, 1)
    two.steps(b, 2)
    torch.cuda.synchronize()
    dt2 = wz.wenozn_workspace_dt(two.ws).item()
    assert dt2 == orc.cfl_dt(orc_problem(orc, p), a.cpu().numpy())
