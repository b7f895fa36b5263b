"""wenozn_rhs_noalloc, the variant for callers that cannot allocate device memory, against
wenozn_rhs on two calls in a row (this file is collected last on purpose)."""
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


@pytest.mark.parametrize("system,nx,ny", [(2, 150, 97), (1, 5000, 1)])
def test_rhs_noalloc_matches_rhs_twice(wz, system, nx, ny):
    p = wz.wenozn_problem_init(system, nx, ny, 1.0 / nx, 1.0 / max(ny, 1))
    ws = wz.workspace(p)
    for call, seed in enumerate((11, 12)):          # two calls in a row, different states
        U0 = inputs.euler2d_ic(nx, ny, seed) if system == 2 else inputs.euler1d_ic(nx, seed)
        U = torch.from_numpy(U0).cuda()
        want = torch.empty_like(U)
        wz.wenozn_rhs(p, U, want, ws)
        got = torch.full_like(U, float("nan"))
        code = wz.lib().wenozn_rhs_noalloc(ctypes.byref(p), ctypes.c_void_p(U.data_ptr()),
                                           ctypes.c_void_p(got.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert code == wz.WENOZN_OK, (call, code)
        torch.cuda.synchronize()
        assert _rel(got, want) <= STEP_TOL, call


def test_rhs_noalloc_rejects_problems_beyond_its_scratch(wz):
    p = wz.wenozn_problem_init(wz.WENOZN_EULER_2D, 1024, 1024, 1e-3, 1e-3)
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = torch.zeros(1, dtype=torch.float64, device="cuda")
    code = wz.lib().wenozn_rhs_noalloc(ctypes.byref(p), ctypes.c_void_p(U.data_ptr()),
                                       ctypes.c_void_p(L.data_ptr()), None)
    assert code == wz.WENOZN_ENOMEM_WS
