"""ctypes front end of the WENO-ZN CPU oracle (``wenozn_oracle.cpp``).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  It shares nothing with the CUDA
library: its own shared object, its own problem struct, its own build line.

Arrays are numpy float64, C-contiguous, laid out as the library lays them out: conserved
variables planar, ``U[nvar][ny][nx]`` with x fastest.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wenozn_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

W_ZN, W_Z, W_LINEAR, W_JS = 0, 1, 2, 3
ADV1D, EULER1D, EULER2D = 0, 1, 2
PERIODIC, OUTFLOW, REFLECTIVE = 0, 1, 2
S_LF, S_LF_FIELD, S_LLF, S_SW = 0, 1, 2, 3      # flux splittings


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain IEEE arithmetic: no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32), ("weights", ctypes.c_int32),
                ("split", ctypes.c_int32), ("pad", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("gamma", ctypes.c_double),
                ("eps", ctypes.c_double), ("A", ctypes.c_double), ("cfl", ctypes.c_double),
                ("adv_speed", ctypes.c_double)]


def problem(system, nx, ny=1, dx=1.0, dy=1.0, bc_x=OUTFLOW, bc_y=OUTFLOW, weights=W_ZN,
            gamma=1.4, eps=1e-40, A=10.0, cfl=0.5, adv_speed=1.0, split=S_LF) -> Problem:
    return Problem(system, nx, ny, bc_x, bc_y, weights, split, 0, dx, dy, gamma, eps, A, cfl, adv_speed)


def nvar(system: int) -> int:
    return {ADV1D: 1, EULER1D: 3, EULER2D: 4}[system]


_D = ctypes.POINTER(ctypes.c_double)
_P = ctypes.POINTER(Problem)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            sig = {
                "oracle_num_threads": (ctypes.c_int, []),
                "oracle_set_num_threads": (None, [ctypes.c_int]),
                "oracle_weno5_parts": (None, [_D, ctypes.c_double, ctypes.c_double, ctypes.c_int, _D]),
                "oracle_reconstruct": (None, [_D, ctypes.c_int64, _D, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int]),
                "oracle_reconstruct_quad": (None, [_D, ctypes.c_int64, _D, ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_double, ctypes.c_int]),
                "oracle_critical_point_error": (ctypes.c_double, [ctypes.c_int, ctypes.c_double,
                                                                  ctypes.c_int, ctypes.c_double, ctypes.c_int]),
                "oracle_fill_ghosts_line": (None, [_D, ctypes.c_int64, ctypes.c_int]),
                "oracle_max_wavespeed": (ctypes.c_double, [_P, _D, ctypes.c_int]),
                "oracle_cfl_dt": (ctypes.c_double, [_P, _D]),
                "oracle_rhs": (None, [_P, _D, _D]),
                "oracle_rk3_step": (ctypes.c_double, [_P, _D, ctypes.c_double, ctypes.c_double]),
                "oracle_run": (ctypes.c_int64, [_P, _D, ctypes.c_double, ctypes.c_double]),
                "oracle_rk3_linear": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double]),
                "oracle_roe_eigen": (None, [_D, _D, ctypes.c_int, ctypes.c_double, _D]),
                "oracle_normal_flux": (None, [_D, ctypes.c_int, ctypes.c_double, _D]),
                "oracle_opcount_rhs": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]),
                "oracle_opcount_rhs_variant": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_int, _D]),
                "oracle_opcount_parts": (None, [ctypes.c_int, _D]),
                "oracle_opcount_parts_variant": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]),
                "oracle_rhs_jvp": (None, [_P, _D, _D, _D, _D]),
                "oracle_steger_warming": (None, [_D, ctypes.c_int, ctypes.c_double, ctypes.c_int, _D]),
                "oracle_field_speed": (ctypes.c_double, [_P, _D, ctypes.c_int, ctypes.c_int]),
                "oracle_rhs_speeds": (None, [_P, _D, _D, _D]),
                "oracle_rhs_jvp_quad": (None, [_P, _D, _D, _D, _D]),
                "oracle_rollout_jvp_quad": (None, [_P, _D, _D, ctypes.c_double, ctypes.c_int64]),
                "oracle_rollout_jvp": (None, [_P, _D, _D, ctypes.c_double, ctypes.c_int64]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_num_threads(n: int) -> None:
    lib().oracle_set_num_threads(int(n))


PART_NAMES = ("q0", "q1", "q2", "IS0", "IS1", "IS2", "tau5", "tau8", "C",
              "alpha0", "alpha1", "alpha2", "omega0", "omega1", "omega2", "fhat")


def weno5_parts(f5, eps=1e-40, A=10.0, kind=W_ZN) -> dict:
    """Every intermediate of one reconstruction f^+_{i+1/2} from f_{i-2..i+2}."""
    f = _f64(f5)
    assert f.shape == (5,)
    out = np.zeros(16)
    lib().oracle_weno5_parts(_ptr(f), eps, A, kind, _ptr(out))
    return dict(zip(PART_NAMES, out.tolist()))


def reconstruct(f_padded, side=+1, eps=1e-40, A=10.0, kind=W_ZN) -> np.ndarray:
    """f^+ (side=+1) or f^- (side=-1) at the n+1 interfaces of a padded line of n+6 values."""
    f = _f64(f_padded)
    n = f.shape[0] - 6
    out = np.zeros(n + 1)
    lib().oracle_reconstruct(_ptr(f), n, _ptr(out), int(side), eps, A, kind)
    return out


def reconstruct_quad(f_padded, side=+1, eps=1e-40, A=10.0, kind=W_ZN) -> np.ndarray:
    """`reconstruct` evaluated in binary128 and rounded to double (no overflow for any input)."""
    f = _f64(f_padded)
    n = f.shape[0] - 6
    out = np.zeros(n + 1)
    lib().oracle_reconstruct_quad(_ptr(f), n, _ptr(out), int(side), eps, A, kind)
    return out


def critical_point_error(k, dx, kind=W_ZN, eps=1e-40, quad=True) -> float:
    return lib().oracle_critical_point_error(int(k), float(dx), int(kind), float(eps), int(bool(quad)))


def fill_ghosts_line(f_padded, bc) -> np.ndarray:
    f = _f64(f_padded).copy()
    lib().oracle_fill_ghosts_line(_ptr(f), f.shape[0] - 6, int(bc))
    return f


def max_wavespeed(P: Problem, U, direction=0) -> float:
    u = _f64(U)
    return lib().oracle_max_wavespeed(ctypes.byref(P), _ptr(u), int(direction))


def cfl_dt(P: Problem, U) -> float:
    u = _f64(U)
    return lib().oracle_cfl_dt(ctypes.byref(P), _ptr(u))


def rhs(P: Problem, U) -> np.ndarray:
    u = _f64(U)
    out = np.zeros_like(u)
    lib().oracle_rhs(ctypes.byref(P), _ptr(u), _ptr(out))
    return out


def rk3_step(P: Problem, U, dt=0.0, t_remaining=0.0):
    """One SSP-RK3 step; returns (U_next, dt_used)."""
    u = _f64(U).copy()
    used = lib().oracle_rk3_step(ctypes.byref(P), _ptr(u), float(dt), float(t_remaining))
    return u, used


def run(P: Problem, U, T, dt=0.0):
    """Advance to time T; returns (U_T, steps)."""
    u = _f64(U).copy()
    steps = lib().oracle_run(ctypes.byref(P), _ptr(u), float(T), float(dt))
    return u, steps


def rk3_linear(lam, dt, u0=1.0) -> float:
    return lib().oracle_rk3_linear(float(lam), float(dt), float(u0))


def roe_eigen(UL, UR, gamma=1.4) -> dict:
    ul, ur = _f64(UL), _f64(UR)
    nv = ul.shape[0]
    out = np.zeros(36)
    lib().oracle_roe_eigen(_ptr(ul), _ptr(ur), nv, gamma, _ptr(out))
    return {"un": out[0], "ut": out[1], "H": out[2], "c": out[3],
            "R": out[4:20].reshape(4, 4)[:nv, :nv].copy(),
            "L": out[20:36].reshape(4, 4)[:nv, :nv].copy()}


def normal_flux(U, gamma=1.4) -> np.ndarray:
    u = _f64(U)
    out = np.zeros(4)
    lib().oracle_normal_flux(_ptr(u), u.shape[0], gamma, _ptr(out))
    return out[: u.shape[0]]


def opcount_rhs(system, nx, ny=1, weights=W_ZN, split=S_LF) -> dict:
    """Algorithmic operation counts of one RHS evaluation on an nx x ny periodic grid."""
    out = np.zeros(5)
    lib().oracle_opcount_rhs_variant(int(system), int(nx), int(ny), int(weights), int(split), _ptr(out))
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), out.tolist()))


def opcount_parts(system, weights=W_ZN, split=S_LF) -> dict:
    """Algorithmic operations (add+mul+div+sqrt) of the pieces of one RHS evaluation."""
    out = np.zeros(9)
    lib().oracle_opcount_parts_variant(int(system), int(weights), int(split), _ptr(out))
    return {"interface": out[0], "cell_per_sweep": out[1], "wavespeed_cell": out[2],
            "difference_cell_per_dir": out[3], "cmp_interface": out[4], "cmp_cell_per_sweep": out[5],
            "cmp_wavespeed_cell": out[6]}


def rhs_jvp(P: Problem, U, dU):
    """(L, J dU) with J the Jacobian of the discrete RHS (forward mode)."""
    u, du = _f64(U), _f64(dU)
    L, dL = np.zeros_like(u), np.zeros_like(u)
    lib().oracle_rhs_jvp(ctypes.byref(P), _ptr(u), _ptr(du), _ptr(L), _ptr(dL))
    return L, dL


def rhs_jvp_quad(P: Problem, U, dU):
    """rhs_jvp evaluated in binary128 (inputs and outputs rounded to double)."""
    u, du = _f64(U), _f64(dU)
    L, dL = np.zeros_like(u), np.zeros_like(u)
    lib().oracle_rhs_jvp_quad(ctypes.byref(P), _ptr(u), _ptr(du), _ptr(L), _ptr(dL))
    return L, dL


def rollout_jvp(P: Problem, U, dU, dt, steps):
    """`steps` fixed-dt SSP-RK3 steps of U and of the tangent dU; returns (U_T, dU_T)."""
    u, du = _f64(U).copy(), _f64(dU).copy()
    lib().oracle_rollout_jvp(ctypes.byref(P), _ptr(u), _ptr(du), float(dt), int(steps))
    return u, du


def rollout_jvp_quad(P: Problem, U, dU, dt, steps):
    """rollout_jvp evaluated in binary128 (inputs and outputs rounded to double)."""
    u, du = _f64(U).copy(), _f64(dU).copy()
    lib().oracle_rollout_jvp_quad(ctypes.byref(P), _ptr(u), _ptr(du), float(dt), int(steps))
    return u, du


def steger_warming(U, sign, gamma=1.4) -> np.ndarray:
    """Steger-Warming F+ (sign > 0) or F- (sign < 0) of one state in the direction frame."""
    u = _f64(U)
    out = np.zeros_like(u)
    lib().oracle_steger_warming(_ptr(u), u.shape[0], gamma, int(sign), _ptr(out))
    return out


def field_speed(P: Problem, U, direction=0, kind=0) -> float:
    """max |lambda_kind| over the grid, kind 0: u_n - c, 1: u_n, 2: u_n + c."""
    u = _f64(U)
    return lib().oracle_field_speed(ctypes.byref(P), _ptr(u), int(direction), int(kind))


def rhs_speeds(P: Problem, U, ax, ay=0.0, fx=(0.0, 0.0, 0.0), fy=(0.0, 0.0, 0.0)) -> np.ndarray:
    """RHS with the LF speeds given instead of computed from U."""
    u = _f64(U)
    sp = _f64([ax, ay, *fx, *fy])
    out = np.zeros_like(u)
    lib().oracle_rhs_speeds(ctypes.byref(P), _ptr(u), _ptr(sp), _ptr(out))
    return out
