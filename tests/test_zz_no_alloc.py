"""wenozn_rhs_noalloc, the variant for callers that cannot allocate device memory, against
wenozn_rhs on two calls in a row (this file is collected last on purpose).

The cases cover the default scheme and the generic paths whose scratch also lives in the
shared array: the per-field LF speeds (cleared by every call), the other weight functions
and the periodic and reflective ghost maps."""
import ctypes

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


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _noalloc(wz, p, U, L):
    return wz.lib().wenozn_rhs_noalloc(ctypes.byref(p), ctypes.c_void_p(U.data_ptr()),
                                       ctypes.c_void_p(L.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


# (system, nx, ny, overrides of the problem)
CASES = [
    (2, 150, 97, {}),
    (1, 5000, 1, {}),
    (0, 3000, 1, {"bc_x": 0}),
    (2, 90, 64, {"split": 1}),                               # per-field LF speeds
    (1, 2000, 1, {"split": 1, "bc_x": 0}),
    (2, 70, 80, {"weights": 1, "bc_x": 0, "bc_y": 2}),       # WENO-Z, periodic x, walls in y
    (1, 1500, 1, {"weights": 3, "eps": 1e-6, "bc_x": 2}),    # Jiang-Shu between walls
    (2, 64, 50, {"split": 2}),                               # local LF
    (1, 1200, 1, {"split": 3}),                              # Steger-Warming
]


@pytest.mark.parametrize("system,nx,ny,over", CASES)
def test_rhs_noalloc_matches_rhs_twice(wz, system, nx, ny, over):
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / max(ny, 1), **over)
    ws = wz.workspace(p)
    for call, seed in enumerate((11, 12)):          # two calls in a row, different states
        if system == 2:
            U0 = inputs.euler2d_ic(nx, ny, seed)
        elif system == 1:
            U0 = inputs.euler1d_ic(nx, seed)
        else:
            U0 = inputs.random_smooth_state(0, nx, 1, seed)
        U = torch.from_numpy(U0).cuda()
        want = torch.empty_like(U)
        wz.wenozn_rhs(p, U, want, ws)
        got = torch.full_like(U, float("nan"))
        code = _noalloc(wz, p, U, got)
        assert code == wz.WENOZN_OK, (call, code)
        torch.cuda.synchronize()
        assert _rel(got, want) <= STEP_TOL, call


def test_rhs_noalloc_rejects_problems_beyond_its_scratch(wz):
    p = wz.wenozn_problem_init(wz.WENOZN_EULER_2D, 1024, 1024, 1e-3, 1e-3)
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(wz, p, U, L) == wz.WENOZN_ENOMEM_WS


def test_rhs_noalloc_is_not_reported_by_last_error(wz):
    """Its status word is the shared array's, not a workspace's: a non-finite state leaves
    wenozn_last_error of the stream untouched."""
    n = 300
    p = wz.wenozn_problem_init(wz.WENOZN_EULER_1D, n, 1, 10.0 / n, 1.0)
    U0 = inputs.euler1d_ic(n, 3)
    U0[0, 0, 7] = np.nan
    U = torch.from_numpy(U0).cuda()
    L = torch.empty_like(U)
    wz.wenozn_last_error()
    assert _noalloc(wz, p, U, L) == wz.WENOZN_OK
    assert wz.wenozn_last_error() == 0
