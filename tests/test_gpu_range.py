"""The reconstruction's range guarantee (wenozn.h, "Range of the reconstruction"): with the
admissible constants, every stencil whose first differences stay below 2^440 gives a finite
result equal to the oracle's plain evaluation of Eq. (new) to rounding, including data whose
division-free weight products leave the double range (large stencils overflow them, data far
below the scale of eps underflow the numerator) and the evaluation falls back to the stencil
rescaled by an exact power of two.

The Euler cases use the self-similarity of the equations: scaling rho, m and E by s leaves
u, c and the LF speed unchanged and scales every flux by s, so for s a large power of two
(eps negligible against the indicators) the oracle's RHS of s U is s times its RHS of U, and
the GPU must match the oracle there; scaled far down, eps dominates the indicators, the
weights turn linear on both sides, and the GPU must still match the oracle."""
import numpy as np
import pytest
import torch

from paper_2004_07954_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def wz():
    from paper_2004_07954_gb300 import build, wenozn
    build.build()
    assert torch.cuda.is_available(), "CUDA device required"
    return wenozn


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


# powers of two from about 1e-200 to 2.2e130 (the largest stencil differences reach 2^437)
SCALE_EXPONENTS = [-664, -498, -398, -332, -199, 0, 66, 86, 93, 100, 199, 332, 433]


def _cases(n, seed):
    g = np.random.default_rng(seed)
    f = g.normal(size=n + 6)
    f[g.random(n + 6) < 0.1] += 5.0
    spike = np.full(n + 6, 0.7)
    spike[n // 3] = -2.0                                        # flat, one spike (IS_0 = IS_2 beside it)
    x = np.linspace(-1, 1, n + 6)
    return [f, np.where(np.arange(n + 6) < n // 2, 0.0, 1.0), spike, np.sin(3 * x) + 0.01 * x ** 3]


@pytest.mark.parametrize("e", SCALE_EXPONENTS)
@pytest.mark.parametrize("weights", [0, 1, 3])
def test_reconstruct_across_the_range(wz, orc, e, weights):
    """Random data with jumps, a pure step, a constant line with one spike and smooth data,
    scaled by 2^e, both sides: finite, and equal to the oracle's binary128 evaluation (which
    cannot overflow) and to its double evaluation wherever that one is finite."""
    eps = 1e-6 if weights == 3 else 1e-40
    n = 600
    for base in _cases(n, abs(e) * 10 + weights):
        f = base * 2.0 ** e
        bound = TOL * np.abs(f).max()
        for side in (1, -1):
            out = torch.empty(n + 1, dtype=torch.float64, device="cuda")
            wz.wenozn_reconstruct_weights(dev(f), out, side, weights, eps=eps)
            got = out.cpu().numpy()
            want = orc.reconstruct_quad(f, side, eps=eps, kind=weights)
            plain = orc.reconstruct(f, side, eps=eps, kind=weights)
            ok = np.isfinite(plain)
            assert np.all(np.isfinite(got)), (e, side)
            assert np.abs(got - want).max() <= bound, (e, side)
            assert np.abs(got[ok] - plain[ok]).max(initial=0.0) <= bound, (e, side)


def test_reconstruct_at_the_stated_bound(wz, orc):
    """First differences just below 2^440 (a step of 1.5 2^439): finite and equal to the
    oracle."""
    n = 64
    f = np.where(np.arange(n + 6) < 30, 0.0, 1.5 * 2.0 ** 439)
    for side in (1, -1):
        out = torch.empty(n + 1, dtype=torch.float64, device="cuda")
        wz.wenozn_reconstruct(dev(f), out, side)
        got = out.cpu().numpy()
        want = orc.reconstruct_quad(f, side)
        assert np.all(np.isfinite(got))
        assert np.abs(got - want).max() <= TOL * np.abs(f).max()


@pytest.mark.parametrize("k", [-900, -400, -120, 90, 130, 250, 400])
@pytest.mark.parametrize("system,nx,ny,bc", [(1, 300, 1, 1), (2, 48, 40, 1), (2, 40, 36, 0)])
def test_euler_rhs_self_similar_scalings(wz, orc, k, system, nx, ny, bc):
    s = 2.0 ** k
    U0 = inputs.euler1d_ic(nx, 4) if system == 1 else inputs.euler2d_ic(nx, ny, 4)
    U = U0 * s
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / ny, bc_x=bc, bc_y=bc)
    P = orc.problem(system, nx, ny, dx=1.0 / nx, dy=1.0 / ny, bc_x=bc, bc_y=bc)
    S = wz.Solver(p)
    got = S.rhs(dev(U)).cpu().numpy()
    want = orc.rhs(P, U)
    assert np.all(np.isfinite(want))
    if k > 0:
        # eps is negligible against the scaled indicators, so the oracle follows the symmetry
        # (scaled far down, eps dominates them and the weights turn linear instead)
        assert np.abs(want - orc.rhs(P, U0) * s).max() <= 1e-13 * np.abs(want).max()
    assert np.all(np.isfinite(got))
    assert np.abs(got - want).max() <= TOL * np.abs(want).max()
    assert S.status() == 0


@pytest.mark.parametrize("k", [-600, 200])
def test_euler2d_step_self_similar(wz, orc, k):
    """One RK3 step of the scaled 2D problem: the same CFL step as the unscaled one, the state
    equal to the oracle's."""
    n = 40
    s = 2.0 ** k
    U = inputs.euler2d_ic(n, n, 6) * s
    p = wz.wenozn_problem_init(2, n, n, 1.0 / n, 1.0 / n)
    P = orc.problem(2, n, n, dx=1.0 / n, dy=1.0 / n)
    S = wz.Solver(p)
    t = dev(U)
    dt = S.step(t, return_dt=True)
    want, dt_o = orc.rk3_step(P, U)
    assert dt == dt_o
    got = t.cpu().numpy()
    assert np.abs(got - want).max() <= TOL * np.abs(want).max()
    assert S.status() == 0


def test_rhs_reports_non_finite_results(wz):
    """Beyond the bound (here 2^500 in a 1D Euler state, where tau8 / eps overflows in any
    evaluation) the RHS is not finite, and the status word says so."""
    n = 200
    U = inputs.euler1d_ic(n, 4) * 2.0 ** 520
    p = wz.wenozn_problem_init(1, n, 1, 10.0 / n, 1.0)
    S = wz.Solver(p)
    L = S.rhs(dev(U)).cpu().numpy()
    if np.all(np.isfinite(L)):
        pytest.skip("finite even here")
    assert S.status() & (1 << wz.WENOZN_ENONFINITE)
