"""The C-ABI library builds, loads without a GPU, exports every entry point the header
declares, and rejects invalid arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wz():
    from paper_2004_07954_gb300 import build, wenozn
    build.build()
    wenozn.lib()
    return wenozn


def declared_entry_points():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(wenozn_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(wz):
    names = declared_entry_points()
    assert len(names) >= 11
    L = wz.lib()
    for n in names:
        assert hasattr(L, n), n


def test_problem_init_defaults(wz):
    p = wz.wenozn_problem_init(wz.WENOZN_EULER_2D, 128, 64, 0.01, 0.02)
    assert (p.nx, p.ny, p.bc_x, p.bc_y, p.flags) == (128, 64, 1, 1, 0)
    assert (p.gamma, p.eps, p.A, p.cfl) == (1.4, 1e-40, 10.0, 0.5)
    p1 = wz.wenozn_problem_init(wz.WENOZN_EULER_1D, 100, 77, 0.1, 0.2)
    assert p1.ny == 1


def test_workspace_size_layout(wz):
    def al(x):
        return (x + 255) // 256 * 256
    p = wz.wenozn_problem_init(wz.WENOZN_EULER_2D, 100, 50, 0.01, 0.02)
    n = 4 * 100 * 50 * 8
    want = 256 + 2 * al(n) + al(4 * 101 * 50 * 8) + al(4 * 100 * 51 * 8)
    assert wz.wenozn_workspace_size(p) == want
    p1 = wz.wenozn_problem_init(wz.WENOZN_EULER_1D, 1000, 1, 0.01, 0)
    assert wz.wenozn_workspace_size(p1) == 256 + 2 * al(3 * 1000 * 8) + al(3 * 1001 * 8)


@pytest.mark.parametrize("field,value", [("nx", 0), ("ny", 0), ("system", 7), ("bc_x", 3), ("dx", 0.0),
                                         ("dx", float("nan")), ("eps", 0.0), ("A", -1.0), ("cfl", 0.0),
                                         ("gamma", 1.0), ("flags", 1), ("eps", 1e-61), ("eps", 2.0),
                                         ("A", 1e-7), ("A", 2e6)])
def test_invalid_problem_rejected_on_host(wz, field, value):
    p = wz.wenozn_problem_init(wz.WENOZN_EULER_2D, 16, 16, 0.1, 0.1)
    setattr(p, field, value)
    n = ctypes.c_size_t(0)
    assert wz.lib().wenozn_workspace_size(ctypes.byref(p), ctypes.byref(n)) == wz.WENOZN_EINVAL
    # null device pointers are rejected before any CUDA call
    assert wz.lib().wenozn_rhs(ctypes.byref(p), None, None, None, 0, None) == wz.WENOZN_EINVAL


def test_null_and_bad_arguments_rejected(wz):
    L = wz.lib()
    assert L.wenozn_reconstruct(None, 10, None, 1, 1e-40, 10.0, None) == wz.WENOZN_EINVAL
    assert L.wenozn_reconstruct(ctypes.c_void_p(256), 0, ctypes.c_void_p(512), 1, 1e-40, 10.0, None) == wz.WENOZN_EINVAL
    assert L.wenozn_reconstruct(ctypes.c_void_p(256), 10, ctypes.c_void_p(512), 0, 1e-40, 10.0, None) == wz.WENOZN_EINVAL
    p = wz.wenozn_problem_init(wz.WENOZN_EULER_1D, 64, 1, 0.1, 0)
    assert L.wenozn_rk3_step(ctypes.byref(p), None, 0.0, 0.0, None, None, 0, None) == wz.WENOZN_EINVAL
    # misaligned workspace
    assert L.wenozn_rk3_step(ctypes.byref(p), ctypes.c_void_p(256), 0.0, 0.0, None,
                             ctypes.c_void_p(257), 1 << 20, None) == wz.WENOZN_EINVAL
    # workspace too small
    assert L.wenozn_rk3_step(ctypes.byref(p), ctypes.c_void_p(256), 0.0, 0.0, None,
                             ctypes.c_void_p(512), 16, None) == wz.WENOZN_ENOMEM_WS
    assert L.wenozn_workspace_status(None, None, 0, None) == wz.WENOZN_EINVAL
    assert L.wenozn_problem_init(None, 0, 1, 1, 1.0, 1.0) == wz.WENOZN_EINVAL


def test_newer_entry_points_reject_bad_arguments_on_host(wz):
    """The chained, keep/reverse, weight-variant and probe entry points check their arguments
    before any CUDA call (so these run without a GPU)."""
    L = wz.lib()
    A = ctypes.c_void_p(256)                       # stand-in device addresses, never touched
    p1 = wz.wenozn_problem_init(wz.WENOZN_EULER_1D, 64, 1, 0.1, 0)
    p2 = wz.wenozn_problem_init(wz.WENOZN_EULER_2D, 16, 16, 0.1, 0.1)
    # chained run: no steps, non-finite dt, no state
    assert L.wenozn_rk3_run(ctypes.byref(p1), A, 0, 0.0, A, 1 << 30, None) == wz.WENOZN_EINVAL
    assert L.wenozn_rk3_run(ctypes.byref(p1), A, 4, float("nan"), A, 1 << 30, None) == wz.WENOZN_EINVAL
    assert L.wenozn_rk3_run(ctypes.byref(p1), None, 4, 0.0, A, 1 << 30, None) == wz.WENOZN_EINVAL
    # keep / reverse segments: 1D default scheme, positive finite dt, at least one step
    for fn in (L.wenozn_rk3_run_keep,):
        assert fn(ctypes.byref(p1), A, A, A, A, 0, 1e-3, A, 1 << 30, None) == wz.WENOZN_EINVAL
        assert fn(ctypes.byref(p1), A, A, A, A, 3, 0.0, A, 1 << 30, None) == wz.WENOZN_EINVAL
        assert fn(ctypes.byref(p2), A, A, A, A, 3, 1e-3, A, 1 << 30, None) == wz.WENOZN_EINVAL
    assert L.wenozn_rk3_vjp_run(ctypes.byref(p1), A, A, A, A, 3, 1e-3, None, A, 1 << 30, None) == wz.WENOZN_EINVAL
    assert L.wenozn_rk3_vjp_run(ctypes.byref(p2), A, A, A, A, 3, 1e-3, A, A, 1 << 30, None) == wz.WENOZN_EINVAL
    # weight variants: unknown weight function, bad side, non-positive eps
    for weights, side, eps in ((4, 1, 1e-40), (-1, 1, 1e-40), (0, 2, 1e-40), (1, 1, 0.0), (0, 1, 1e-61),
                               (3, 1, 1.5)):
        assert L.wenozn_reconstruct_weights(A, 10, A, side, weights, eps, 10.0, None) == wz.WENOZN_EINVAL
    # the constant A of Eq. (function) outside [1e-6, 1e6]
    for a in (0.0, 1e-7, 1e7):
        assert L.wenozn_reconstruct(A, 10, A, 1, 1e-40, a, None) == wz.WENOZN_EINVAL
    # host-buffer step and CFL step: no state, no staging buffer, no workspace
    h = (ctypes.c_double * 64)()
    assert L.wenozn_rk3_step_host(ctypes.byref(p1), None, h, A, 0.0, 0.0, None, A, 1 << 30, None) == wz.WENOZN_EINVAL
    assert L.wenozn_rk3_step_host(ctypes.byref(p1), h, h, None, 0.0, 0.0, None, A, 1 << 30, None) == wz.WENOZN_EINVAL
    assert L.wenozn_rk3_step_host(ctypes.byref(p1), h, h, A, float("nan"), 0.0, None, A, 1 << 30, None) == \
        wz.WENOZN_EINVAL
    assert L.wenozn_rk3_step_host(ctypes.byref(p1), h, h, A, 0.0, 0.0, None, A, 16, None) == wz.WENOZN_ENOMEM_WS
    assert L.wenozn_cfl_dt(ctypes.byref(p1), None, None, A, 1 << 30, None) == wz.WENOZN_EINVAL
    hp = (ctypes.c_void_p * 2)(ctypes.cast(h, ctypes.c_void_p), None)
    ok = (ctypes.c_void_p * 2)(ctypes.cast(h, ctypes.c_void_p), ctypes.cast(h, ctypes.c_void_p))
    B_ = ctypes.c_void_p(512)
    for count, ins, d0, d1 in ((0, ok, A, B_), (2, hp, A, B_), (2, ok, A, A), (2, ok, None, B_)):
        assert L.wenozn_rk3_stream_host(ctypes.byref(p1), count, ins, ok, d0, d1, 0.0, A, 1 << 30, None, None,
                                        None) == wz.WENOZN_EINVAL
    assert L.wenozn_cfl_dt(ctypes.byref(p1), A, None, ctypes.c_void_p(257), 1 << 30, None) == wz.WENOZN_EINVAL
    # FP64 rate probe: sizes outside [4, 2^32], no result pointer
    g = ctypes.c_double(0.0)
    for bad in (0, 3, (1 << 32) + 1):
        assert L.wenozn_fp64_fma_rate(bad, ctypes.byref(g), None) == wz.WENOZN_EINVAL
    assert L.wenozn_fp64_fma_rate(1 << 10, None, None) == wz.WENOZN_EINVAL


def test_flux_directions_checked_on_host(wz):
    """wenozn_flux: direction 0 for every system, 1 and 2 (both sweeps in one launch) for 2D
    Euler only, a speed array required except for advection; flux_shape gives the layout of
    each direction (direction 2: the x fluxes then the y fluxes, one flat array)."""
    L = wz.lib()
    A, B = ctypes.c_void_p(256), ctypes.c_void_p(1 << 20)
    p0 = wz.wenozn_problem_init(wz.WENOZN_ADVECTION_1D, 64, 1, 0.1, 0)
    p1 = wz.wenozn_problem_init(wz.WENOZN_EULER_1D, 64, 1, 0.1, 0)
    p2 = wz.wenozn_problem_init(wz.WENOZN_EULER_2D, 16, 12, 0.1, 0.1)
    for p in (p0, p1):
        for d in (1, 2, -1, 3):
            assert L.wenozn_flux(ctypes.byref(p), A, A, d, B, None) == wz.WENOZN_EINVAL
    for d in (-1, 3):
        assert L.wenozn_flux(ctypes.byref(p2), A, A, d, B, None) == wz.WENOZN_EINVAL
    assert L.wenozn_flux(ctypes.byref(p2), A, None, 2, B, None) == wz.WENOZN_EINVAL     # no speeds
    assert L.wenozn_flux(ctypes.byref(p2), A, A, 2, A, None) == wz.WENOZN_EINVAL        # Fout == U
    assert L.wenozn_flux(ctypes.byref(p2), A, A, 2, None, None) == wz.WENOZN_EINVAL
    assert wz.flux_shape(p2, 0) == (4, 12, 17)
    assert wz.flux_shape(p2, 1) == (4, 13, 16)
    assert wz.flux_shape(p2, 2) == (4 * 12 * 17 + 4 * 13 * 16,)


def test_status_strings_and_version(wz):
    for code in range(6):
        assert wz.wenozn_status_string(code)
    assert wz.wenozn_status_string(99) == "unknown status"
    assert re.fullmatch(r"\d+\.\d+\.\d+", wz.wenozn_version())


def test_oracle_and_library_share_no_code():
    """The oracle and the CUDA path are independent: neither includes, imports or links the
    other, and only the seeded-input module is common to their callers."""
    csrc = os.path.join(ROOT, "paper_2004_07954_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text).lower() or f == "inputs.py", f
    otext = open(os.path.join(ROOT, "oracle", "wenozn_oracle.cpp")).read()
    assert "wenozn.h" not in otext and "csrc" not in otext
    assert "paper_2004_07954_gb300" not in open(os.path.join(ROOT, "oracle", "oracle.py")).read()
