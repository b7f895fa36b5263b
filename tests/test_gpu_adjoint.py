"""Discrete adjoint kernels against the oracle's forward-mode derivatives and against
central finite differences."""
import numpy as np
import pytest
import torch

from paper_2004_07954_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wz():
    from paper_2004_07954_gb300 import build, wenozn
    build.build()
    assert torch.cuda.is_available(), "CUDA device required"
    return wenozn


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _problem(wz, orc, system, n, dx, bc):
    p = wz.wenozn_problem_init(system, n, 1, dx, 1.0, bc_x=bc)
    P = orc.problem(system, n, 1, dx=dx, bc_x=bc)
    return p, P


def _state(system, n, seed):
    return inputs.random_smooth_state(system, n, 1, seed)


@pytest.mark.parametrize("system,bc,n", [(1, 1, 12), (1, 0, 12), (0, 0, 12), (1, 1, 3), (1, 0, 2), (0, 0, 5),
                                         (1, 1, 1)])
def test_rhs_vjp_elementwise_against_oracle_jacobian(wz, orc, system, bc, n):
    """Full Jacobian of the oracle RHS from forward-mode columns; J^T lam from the GPU
    (small grids exercise the ghost-cell preimages of the gather)."""
    p, P = _problem(wz, orc, system, n, 0.1, bc)
    U = _state(system, n, seed=3)
    nv = U.shape[0]
    J = np.zeros((nv * n, nv * n))
    for col in range(nv * n):
        e = np.zeros(nv * n)
        e[col] = 1.0
        _, dL = orc.rhs_jvp(P, U, e.reshape(U.shape))
        J[:, col] = dL.ravel()
    lam = np.random.default_rng(1).normal(size=U.shape)
    out = torch.empty_like(dev(U))
    ws = wz.vjp_workspace(p)
    wz.wenozn_rhs_vjp(p, dev(U), dev(lam), out, ws)
    want = (J.T @ lam.ravel()).reshape(U.shape)
    # relative to the scale of the summed terms (lam / dx times O(1) flux derivatives): on
    # one cell both interfaces see the same stencil, the RHS vanishes identically and only
    # the cancellation residue of those terms remains
    scale = max(np.abs(want).max(), np.abs(lam).max() / 0.1)
    assert np.abs(out.cpu().numpy() - want).max() <= 1e-10 * scale


@pytest.mark.parametrize("system,n,bc", [(1, 300, 1), (1, 257, 0), (0, 500, 0), (1, 4099, 1),
                                         (1, 12289, 0), (1, 65536, 1)])
def test_rhs_vjp_dot_product(wz, orc, system, n, bc):
    """(Lines of 10240 cells and more take the one-thread-per-interface stage kernel.)"""
    p, P = _problem(wz, orc, system, n, 10.0 / n, bc)
    U = inputs.euler1d_ic(n, seed=4) if system == 1 else _state(0, n, 4)
    g = np.random.default_rng(2)
    ws = wz.vjp_workspace(p)
    for _ in range(3):
        v, lam = g.normal(size=U.shape), g.normal(size=U.shape)
        # binary128 reference: the double forward-mode derivative of C divides by
        # (tau5 + eps)^2 and loses digits where IS_0 ~ IS_2 (e.g. the exact antisymmetry of
        # the sine profile about x = 0, a cell centre for n = 257 and n = 4099)
        _, Jv = orc.rhs_jvp_quad(P, U, v)
        out = torch.empty_like(dev(U))
        wz.wenozn_rhs_vjp(p, dev(U), dev(lam), out, ws)
        a, b = float(np.sum(lam * Jv)), float(np.sum(out.cpu().numpy() * v))
        assert b == pytest.approx(a, rel=1e-10, abs=1e-12 * np.abs(lam).sum() * np.abs(Jv).max())


@pytest.mark.parametrize("system,bc,n", [(1, 0, 240), (1, 1, 240), (0, 0, 240), (1, 0, 16384), (1, 1, 16384)])
def test_rk3_step_vjp_dot_product(wz, orc, system, bc, n):
    """One RK3 step of the smooth adjoint workload (no rounding-flat fields, whose exact
    tangent is noise-driven with eps = 1e-40); 16384 cells take the one-thread-per-interface
    stage kernel."""
    p, P = _problem(wz, orc, system, n, 10.0 / n, bc)
    U = inputs.adjoint_ic(n, seed=6) if system == 1 else _state(0, n, 6)
    dt = 0.4 * p.dx / (orc.max_wavespeed(P, U) if system == 1 else 1.0)
    g = np.random.default_rng(3)
    ws = wz.vjp_workspace(p)
    for _ in range(3):
        v, lam = g.normal(size=U.shape), g.normal(size=U.shape)
        _, Jv = orc.rollout_jvp_quad(P, U, v, dt, 1)      # binary128 reference (see above)
        l = dev(lam)
        wz.wenozn_rk3_step_vjp(p, dev(U), dt, l, ws)
        a, b = float(np.sum(lam * Jv)), float(np.sum(l.cpu().numpy() * v))
        assert b == pytest.approx(a, rel=1e-10)


@pytest.mark.parametrize("system,bc", [(1, 0), (1, 1), (0, 0)])
def test_rk3_step_vjp_from_stored_stages_is_bit_identical(wz, system, bc):
    """The reverse step fed with the forward step's stored stage inputs and LF speeds equals
    the reverse step that recomputes them, bit for bit."""
    n = 1000
    p = wz.wenozn_problem_init(system, n, 1, 10.0 / n, 1.0, bc_x=bc)
    U = dev(inputs.adjoint_ic(n, seed=14) if system == 1 else _state(0, n, 14))
    dt = 0.3 * p.dx
    lam = dev(np.random.default_rng(5).normal(size=tuple(U.shape)))
    ws = wz.vjp_workspace(p)
    l1 = lam.clone()
    wz.wenozn_rk3_step_vjp(p, U, dt, l1, ws)
    U1n = U.clone()
    wz.wenozn_rk3_step(p, U1n, ws, dt=dt)
    S1, S2, A = (t.clone() for t in wz.workspace_stages(p, ws))
    l2 = lam.clone()
    wz.wenozn_rk3_step_vjp_stages(p, U, S1, S2, A, dt, l2, ws)
    assert torch.equal(l1, l2)
    with pytest.raises(wz.WenoznError):
        wz.wenozn_rk3_step_vjp_stages(p, U, S1, S2, A, dt, S1, ws)


@pytest.mark.parametrize("system,bc", [(1, 0), (1, 1), (0, 0)])
def test_rk3_step_keep_matches_in_place_step(wz, system, bc):
    """The out-of-place step that keeps its stage inputs gives the in-place step's state,
    stage buffers and LF speeds bit for bit, and leaves its input untouched."""
    n = 777
    p = wz.wenozn_problem_init(system, n, 1, 10.0 / n, 1.0, bc_x=bc)
    U = dev(inputs.adjoint_ic(n, seed=15) if system == 1 else _state(0, n, 15))
    U0 = U.clone()
    dt = 0.3 * p.dx
    ws = wz.vjp_workspace(p)
    Un, S1, S2 = torch.empty_like(U), torch.empty_like(U), torch.empty_like(U)
    A = torch.empty(3, dtype=torch.float64, device="cuda")
    wz.wenozn_rk3_step_keep(p, U, Un, dt, S1, S2, A, ws)
    assert torch.equal(U, U0)
    V = U.clone()
    wz.wenozn_rk3_step(p, V, ws, dt=dt)
    W1, W2, WA = wz.workspace_stages(p, ws)
    assert torch.equal(Un, V) and torch.equal(S1, W1) and torch.equal(S2, W2) and torch.equal(A, WA)
    with pytest.raises(wz.WenoznError):
        wz.wenozn_rk3_step_keep(p, U, U, dt, S1, S2, A, ws)


@pytest.mark.parametrize("n", [640, 20000])
def test_chained_keep_and_reverse_equal_the_single_steps(wz, n):
    """wenozn_rk3_run_keep / wenozn_rk3_vjp_run against wenozn_rk3_step_keep /
    wenozn_rk3_step_vjp_stages step by step, bit for bit (both forms of the stage kernel)."""
    m = 9
    p = wz.wenozn_problem_init(1, n, 1, 10.0 / n, 1.0, bc_x=0)
    U0 = dev(inputs.adjoint_ic(n, seed=16))
    dt = 0.3 * p.dx
    ws = wz.vjp_workspace(p)
    X = torch.empty((m + 1,) + tuple(U0.shape), dtype=torch.float64, device="cuda")
    S1, S2 = torch.empty_like(X[:m]), torch.empty_like(X[:m])
    A = torch.empty(3 * m + 1, dtype=torch.float64, device="cuda")
    X[0].copy_(U0)
    wz.wenozn_rk3_run_keep(p, X, S1, S2, A, m, dt, ws)
    U = U0.clone()
    T1, T2 = torch.empty_like(U), torch.empty_like(U)
    Ak = torch.empty(3, dtype=torch.float64, device="cuda")
    for k in range(m):
        Un = torch.empty_like(U)
        wz.wenozn_rk3_step_keep(p, U, Un, dt, T1, T2, Ak, ws)
        assert torch.equal(X[k], U) and torch.equal(S1[k], T1) and torch.equal(S2[k], T2)
        assert torch.equal(A[3 * k:3 * k + 3], Ak)
        U = Un
    assert torch.equal(X[m], U)
    lam0 = dev(np.random.default_rng(8).normal(size=tuple(U0.shape)))
    l1, l2 = lam0.clone(), lam0.clone()
    wz.wenozn_rk3_vjp_run(p, X, S1, S2, A, m, dt, l1, ws)
    for k in reversed(range(m)):
        wz.wenozn_rk3_step_vjp_stages(p, X[k], S1[k], S2[k], A[3 * k:3 * k + 3], dt, l2, ws)
    assert torch.equal(l1, l2)


def test_chained_reverse_is_repeatable_at_the_benchmark_size(wz):
    """N = 8192, 150 steps: three runs of the chained reverse (one call, programmatically
    dependent launches) and the step-by-step reverse agree bit for bit."""
    n, m = 8192, 150
    p = wz.wenozn_problem_init(1, n, 1, 10.0 / n, 1.0, bc_x=0)
    U0 = dev(inputs.adjoint_ic(n, seed=3))
    dt = 0.4 * p.dx
    ws = wz.vjp_workspace(p)
    X = torch.empty((m + 1,) + tuple(U0.shape), dtype=torch.float64, device="cuda")
    S1, S2 = torch.empty_like(X[:m]), torch.empty_like(X[:m])
    A = torch.empty(3 * m + 1, dtype=torch.float64, device="cuda")
    X[0].copy_(U0)
    wz.wenozn_rk3_run_keep(p, X, S1, S2, A, m, dt, ws)
    lam0 = dev(np.random.default_rng(5).normal(size=tuple(U0.shape)))
    runs = []
    for _ in range(3):
        lam = lam0.clone()
        wz.wenozn_rk3_vjp_run(p, X, S1, S2, A, m, dt, lam, ws)
        runs.append(lam)
    step = lam0.clone()
    for k in reversed(range(m)):
        wz.wenozn_rk3_step_vjp_stages(p, X[k], S1[k], S2[k], A[3 * k:3 * k + 3], dt, step, ws)
    for r in runs:
        assert torch.equal(r, runs[0])
    assert torch.equal(step, runs[0])


def _wave_speeds(U, gamma=1.4):
    rho, m, E = U[0, 0], U[1, 0], U[2, 0]
    u = m / rho
    return np.abs(u) + np.sqrt(gamma * (gamma - 1.0) * (E - 0.5 * m * u) / rho)


@pytest.mark.parametrize("n,bc,target", [(200, 1, 0), (200, 1, 199), (200, 1, 26), (200, 1, 27), (200, 1, 29),
                                         (200, 0, 1), (200, 0, 198), (200, 0, 54),
                                         (20000, 1, 0), (20000, 1, 19999), (20000, 1, 58), (20000, 1, 59),
                                         (20000, 0, 1), (20000, 0, 19998), (20000, 0, 118)])
def test_reverse_with_the_lf_argmax_at_a_correction_target(wz, orc, n, bc, target):
    """The LF speed's argmax planted (a one-cell pressure spike that holds it through every
    stage input) at a cell the deferred corrections touch: a ghost-cell target at either
    boundary (outflow: cells 0, n-1; periodic: 0..2, n-3..n-1), or a cell in the windows of
    two neighbouring blocks (n = 200, per-field kernel, 27 owned cells a block: 24..29 and
    51..56 lie in two; n = 20000, one-thread-per-interface kernel, 59 owned cells: 56..61 and
    115..120).  Two reverse steps in one chained call (six stage launches: every pending slot
    is read) against the oracle's binary128 forward-mode derivative, and bit for bit against
    the step-by-step reverse (each call completing in place)."""
    m = 2
    p, P = _problem(wz, orc, 1, n, 10.0 / n, bc)
    W = inputs.adjoint_ic(n, seed=9)
    rho, mom = W[0, 0], W[1, 0]
    u = mom / rho
    pr = 0.4 * (W[2, 0] - 0.5 * mom * u)
    pr[target] *= 1.8
    U0 = inputs.cons_from_prim(rho, u, pr).reshape(3, 1, n).copy()
    dt = 0.1 * p.dx / orc.max_wavespeed(P, U0)
    ws = wz.vjp_workspace(p)
    X = torch.empty((m + 1,) + tuple(U0.shape), dtype=torch.float64, device="cuda")
    S1, S2 = torch.empty_like(X[:m]), torch.empty_like(X[:m])
    A = torch.empty(3 * m + 1, dtype=torch.float64, device="cuda")
    X[0].copy_(dev(U0))
    wz.wenozn_rk3_run_keep(p, X, S1, S2, A, m, dt, ws)
    for k in range(m):                                    # the planted argmax holds
        for st in (X[k], S1[k], S2[k]):
            assert int(np.argmax(_wave_speeds(st.cpu().numpy()))) == target
    g = np.random.default_rng(11)
    for _ in range(2):
        v, lam = g.normal(size=U0.shape), g.normal(size=U0.shape)
        _, Jv = orc.rollout_jvp_quad(P, U0, v, dt, m)
        l1, l2 = dev(lam), dev(lam)
        wz.wenozn_rk3_vjp_run(p, X, S1, S2, A, m, dt, l1, ws)
        for k in reversed(range(m)):
            wz.wenozn_rk3_step_vjp_stages(p, X[k], S1[k], S2[k], A[3 * k:3 * k + 3], dt, l2, ws)
        assert torch.equal(l1, l2)
        a, b = float(np.sum(lam * Jv)), float(np.sum(l1.cpu().numpy() * v))
        assert b == pytest.approx(a, rel=1e-10)


def _loss_grad(wz, p, U0, dt, steps, target, every=1):
    from paper_2004_07954_gb300.rollout import rollout
    U = dev(U0).requires_grad_(True)
    UT = rollout(U, p, dt, steps, checkpoint_every=every)
    loss = 0.5 * ((UT[0] - target) ** 2).sum()
    (g,) = torch.autograd.grad(loss, U)
    return float(loss.item()), g.cpu().numpy()


def test_rollout_gradient_against_oracle_jvp(wz, orc):
    """Adjoint of a 30-step rollout of the smooth adjoint workload against the oracle's
    forward-mode derivative (the CPU reference gradient along seeded directions)."""
    n, steps = 200, 30
    p, P = _problem(wz, orc, 1, n, 10.0 / n, 0)
    U0 = inputs.adjoint_ic(n, seed=7)
    dt = 0.5 * p.dx / orc.max_wavespeed(P, U0)
    target = dev(inputs.adjoint_ic(n, seed=8)[0])
    loss, grad = _loss_grad(wz, p, U0, dt, steps, target)
    UT, _ = orc.rollout_jvp(P, U0, np.zeros_like(U0), dt, steps)
    resid = UT[0] - target.cpu().numpy()
    g = np.random.default_rng(4)
    for _ in range(5):
        v = g.normal(size=U0.shape)
        _, dUT = orc.rollout_jvp_quad(P, U0, v, dt, steps)
        want = float(np.sum(resid * dUT[0]))
        assert float(np.sum(grad * v)) == pytest.approx(want, rel=1e-8)


def test_rollout_gradient_against_central_fd(wz, orc):
    """Central differences (h = 1e-7) of the GPU forward on seeded directions."""
    from paper_2004_07954_gb300.rollout import rollout
    n, steps, h = 512, 200, 1e-7
    p, P = _problem(wz, orc, 1, n, 10.0 / n, 0)
    U0 = inputs.adjoint_ic(n, seed=9)
    dt = 0.5 * p.dx / orc.max_wavespeed(P, U0)
    target = dev(inputs.adjoint_ic(n, seed=10)[0])
    _, grad = _loss_grad(wz, p, U0, dt, steps, target)

    def loss_at(U):
        with torch.no_grad():
            UT = rollout(dev(U), p, dt, steps)
            return 0.5 * float(((UT[0] - target) ** 2).sum().item())
    g = np.random.default_rng(11)
    for _ in range(6):
        v = g.normal(size=U0.shape) * np.abs(U0)          # relative perturbation direction
        fd = (loss_at(U0 + h * v) - loss_at(U0 - h * v)) / (2 * h)
        assert float(np.sum(grad * v)) == pytest.approx(fd, rel=1e-6)


def test_checkpoint_interval_does_not_change_the_gradient(wz, orc):
    n, steps = 256, 23
    p, P = _problem(wz, orc, 1, n, 10.0 / n, 0)
    U0 = inputs.adjoint_ic(n, seed=12)
    dt = 0.5 * p.dx / orc.max_wavespeed(P, U0)
    target = dev(inputs.adjoint_ic(n, seed=13)[0])
    _, g1 = _loss_grad(wz, p, U0, dt, steps, target, every=1)
    _, g7 = _loss_grad(wz, p, U0, dt, steps, target, every=7)
    _, g50 = _loss_grad(wz, p, U0, dt, steps, target, every=50)
    assert np.array_equal(g1, g7) and np.array_equal(g1, g50)


def test_vjp_rejects_2d(wz):
    p = wz.wenozn_problem_init(wz.WENOZN_EULER_2D, 8, 8, 0.1, 0.1)
    with pytest.raises(wz.WenoznError):
        wz.wenozn_vjp_workspace_size(p)
