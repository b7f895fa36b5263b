"""Batched ragged 1D Euler (one persistent launch per RK stage) against the oracle run on
each instance separately."""
import numpy as np
import pytest
import torch

from paper_2004_07954_gb300 import inputs

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12


@pytest.fixture(scope="module")
def wz():
    from paper_2004_07954_gb300 import build, wenozn
    build.build()
    assert torch.cuda.is_available(), "CUDA device required"
    return wenozn


def _batch(B, seed, n_min, n_max):
    sizes, offsets, U = inputs.euler1d_batch(B, seed, n_min, n_max)
    dx = 10.0 / sizes
    return sizes, offsets, dx, U


def _oracle_steps(orc, U0, offsets, dx, steps, t_final=0.0):
    out, dts = np.empty_like(U0), []
    for b in range(offsets.size - 1):
        n = int(offsets[b + 1] - offsets[b])
        P = orc.problem(orc.EULER1D, n, 1, dx=float(dx[b]))
        u = U0[:, offsets[b]:offsets[b + 1]].reshape(3, 1, n).copy()
        t, used = 0.0, 0.0
        for _ in range(steps):
            if t_final > 0 and t >= t_final:
                used = 0.0
                continue
            u, used = orc.rk3_step(P, u, 0.0, (t_final - t) if t_final > 0 else 0.0)
            t += used
        out[:, offsets[b]:offsets[b + 1]] = u[:, 0, :]
        dts.append(used)
    return out, np.array(dts)


def _rel_per_instance(got, want, offsets):
    worst = 0.0
    for b in range(offsets.size - 1):
        g, w = got[:, offsets[b]:offsets[b + 1]], want[:, offsets[b]:offsets[b + 1]]
        worst = max(worst, np.abs(g - w).max() / np.abs(w).max())
    return worst


def test_batch_parity_every_shape(wz, orc):
    sizes, offsets, dx, U0 = _batch(12, seed=3, n_min=20, n_max=1500)
    want, dts = _oracle_steps(orc, U0, offsets, dx, 3)
    _, dts1 = _oracle_steps(orc, U0, offsets, dx, 1)
    results = []
    for shape in range(wz.wenozn_batch_num_shapes()):
        U = torch.from_numpy(U0.copy()).cuda()
        bt = wz.Batch(offsets, dx, U, shape=shape)
        bt.step(U)
        # the first CFL step comes from identical data: bit-exact; later ones from states
        # that differ by rounding
        assert np.array_equal(bt.steps_taken().cpu().numpy(), dts1)
        bt.step(U)
        bt.step(U)
        got = U.cpu().numpy()
        assert _rel_per_instance(got, want, offsets) <= STEP_TOL, shape
        assert bt.steps_taken().cpu().numpy() == pytest.approx(dts, rel=1e-12)
        assert bt.status() == 0
        results.append(got)
    for r in results[1:]:
        assert np.array_equal(r, results[0])                                # tile shape changes nothing


def test_batch_single_and_tiny_instances(wz, orc):
    offsets = np.array([0, 1, 3, 9, 700, 701], dtype=np.int64)
    g = np.random.default_rng(5)
    U0 = np.concatenate([inputs.random_smooth_state(1, int(offsets[b + 1] - offsets[b]), 1, seed=b)[:, 0, :]
                         for b in range(5)], axis=1)
    dx = g.uniform(0.01, 0.1, size=5)
    want, _ = _oracle_steps(orc, U0, offsets, dx, 2)
    U = torch.from_numpy(U0.copy()).cuda()
    bt = wz.Batch(offsets, dx, U)
    bt.step(U)
    bt.step(U)
    assert _rel_per_instance(U.cpu().numpy(), want, offsets) <= STEP_TOL


def test_batch_t_final_clips_each_instance(wz, orc):
    sizes, offsets, dx, U0 = _batch(6, seed=9, n_min=50, n_max=400)
    t_final = 0.02
    want, _ = _oracle_steps(orc, U0, offsets, dx, 40, t_final)
    U = torch.from_numpy(U0.copy()).cuda()
    bt = wz.Batch(offsets, dx, U, t_final=t_final)
    for _ in range(40):
        bt.step(U)
    assert np.all(bt.times().cpu().numpy() == pytest.approx(t_final, rel=1e-14))
    assert _rel_per_instance(U.cpu().numpy(), want, offsets) <= 1e-10


def test_batch_graph_replay_matches_eager(wz):
    sizes, offsets, dx, U0 = _batch(64, seed=1, n_min=128, n_max=4096)
    Ue = torch.from_numpy(U0.copy()).cuda()
    be = wz.Batch(offsets, dx, Ue)
    for _ in range(6):
        be.step(Ue)
    Ug = torch.from_numpy(U0.copy()).cuda()
    bg = wz.Batch(offsets, dx, Ug)
    graph = bg.capture(Ug, 3)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(Ue, Ug)
    assert torch.equal(be.times(), bg.times())


def test_batch_tuner_picks_a_shape(wz):
    sizes, offsets, dx, U0 = _batch(32, seed=2, n_min=128, n_max=8192)
    U = torch.from_numpy(U0).cuda()
    bt = wz.Batch(offsets, dx, U)
    ms = bt.tune(U.clone(), steps=1)
    assert len(ms) == wz.wenozn_batch_num_shapes() and all(m > 0 for m in ms)
    assert bt.bp.shape == int(np.argmin(ms))


def test_batch_full_size_sampled(wz, orc):
    """2048 instances, sizes log-uniform in [128, 16384] (about 6.9 M cells), one RK3 step
    with the default shape; 24 instances (smallest, largest, random) against the oracle."""
    sizes, offsets, dx, U0 = _batch(2048, seed=0, n_min=128, n_max=16384)
    U = torch.from_numpy(U0.copy()).cuda()
    bt = wz.Batch(offsets, dx, U)
    bt.step(U)
    got = U.cpu().numpy()
    dts = bt.steps_taken().cpu().numpy()
    g = np.random.default_rng(0)
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes)), *g.choice(2048, 22, replace=False).tolist()}
    for b in sorted(picks):
        n = int(sizes[b])
        P = orc.problem(orc.EULER1D, n, 1, dx=float(dx[b]))
        u, used = orc.rk3_step(P, U0[:, offsets[b]:offsets[b + 1]].reshape(3, 1, n))
        assert dts[b] == used
        w = u[:, 0, :]
        assert np.abs(got[:, offsets[b]:offsets[b + 1]] - w).max() <= STEP_TOL * np.abs(w).max(), b
    assert bt.status() == 0


def test_batch_tuning_table_is_consulted(wz):
    """A tuned size class is remembered for the process: another batch of the same class (same
    boundary and instance sizes, other data) steps with the tuned shape and, asked to tune with
    steps = 0, takes it without timing; a batch of another class keeps the default."""
    sizes, offsets, dx, U0 = _batch(40, seed=21, n_min=100, n_max=900)
    periodic = wz.WENOZN_BC_PERIODIC
    U = torch.from_numpy(U0.copy()).cuda()
    a = wz.Batch(offsets, dx, U, bc=periodic)
    assert a.shape_in_use() == 3                      # the default: nothing tuned for this class yet
    a.tune(U.clone(), steps=1)
    chosen = a.bp.shape
    other = np.concatenate([inputs.euler1d_ic(int(n), 500 + b)[:, 0, :] for b, n in enumerate(sizes)], axis=1)
    V = torch.from_numpy(other).cuda()
    b = wz.Batch(offsets, dx, V, bc=periodic)
    assert b.bp.shape == -1 and b.shape_in_use() == chosen
    ms = b.tune(V.clone(), steps=0)
    assert b.bp.shape == chosen and all(m == 0.0 for m in ms)
    W = V.clone()
    b.bp.shape = -1
    b.step(V)                                         # the table's shape ...
    c = wz.Batch(offsets, dx, W, bc=periodic, shape=chosen)
    c.step(W)                                         # ... is the explicit one
    assert torch.equal(V, W)
    d = wz.Batch(offsets, dx, W.clone(), bc=wz.WENOZN_BC_OUTFLOW)
    assert d.shape_in_use() == 3
