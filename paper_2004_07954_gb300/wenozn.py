"""Thin Python binding of libwenozn.so (ctypes).

Argument marshalling only: every step of the solver runs in the library's CUDA kernels.
Device buffers are torch tensors (float64, CUDA, C-contiguous); streams default to torch's
current stream.  If the shared library is missing or cannot be loaded the first call
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libwenozn.so")

WENOZN_OK, WENOZN_EINVAL, WENOZN_ECUDA, WENOZN_ENOMEM_WS, WENOZN_ENONFINITE, WENOZN_ETIMEOUT = range(6)
WENOZN_BC_PERIODIC, WENOZN_BC_OUTFLOW, WENOZN_BC_REFLECTIVE = 0, 1, 2
WENOZN_WEIGHTS_ZN, WENOZN_WEIGHTS_Z, WENOZN_WEIGHTS_LINEAR, WENOZN_WEIGHTS_JS = 0, 1, 2, 3
WENOZN_SPLIT_LF, WENOZN_SPLIT_LF_FIELD, WENOZN_SPLIT_LLF, WENOZN_SPLIT_SW = 0, 1, 2, 3
WENOZN_ADVECTION_1D, WENOZN_EULER_1D, WENOZN_EULER_2D = 0, 1, 2
NVAR = {WENOZN_ADVECTION_1D: 1, WENOZN_EULER_1D: 3, WENOZN_EULER_2D: 4}


class WenoznError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        super().__init__(f"{fn}: {wenozn_status_string(code)} (status {code})")


class wenozn_problem(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32), ("weights", ctypes.c_int32),
                ("split", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("gamma", ctypes.c_double),
                ("eps", ctypes.c_double), ("A", ctypes.c_double), ("cfl", ctypes.c_double),
                ("adv_speed", ctypes.c_double)]

    @property
    def nvar(self) -> int:
        return NVAR[self.system]

    @property
    def shape(self):
        return (self.nvar, self.ny, self.nx)


class wenozn_batch_params(ctypes.Structure):
    _fields_ = [("nbatch", ctypes.c_int32), ("bc", ctypes.c_int32), ("shape", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("gamma", ctypes.c_double), ("eps", ctypes.c_double),
                ("A", ctypes.c_double), ("cfl", ctypes.c_double), ("t_final", ctypes.c_double)]


_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_P = ctypes.POINTER(wenozn_problem)
_SIGNATURES = {
    "wenozn_problem_init": [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double],
    "wenozn_workspace_size": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "wenozn_fill_ghosts": [_P, _VP, _VP],
    "wenozn_reconstruct": [_VP, ctypes.c_int64, _VP, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _VP],
    "wenozn_reconstruct_weights": [_VP, ctypes.c_int64, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                   ctypes.c_double, _VP],
    "wenozn_max_wavespeed": [_P, _VP, _VP, _VP, _VP],
    "wenozn_flux": [_P, _VP, _VP, ctypes.c_int32, _VP, _VP],
    "wenozn_rhs": [_P, _VP, _VP, _VP, ctypes.c_size_t, _VP],
    "wenozn_rhs_noalloc": [_P, _VP, _VP, _VP],
    "wenozn_rk3_step": [_P, _VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                        _VP, ctypes.c_size_t, _VP],
    "wenozn_rk3_step_host": [_P, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                             _VP, ctypes.c_size_t, _VP],
    "wenozn_cfl_dt": [_P, _VP, ctypes.POINTER(ctypes.c_double), _VP, ctypes.c_size_t, _VP],
    "wenozn_rk3_stream_host": [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                               _VP, _VP, ctypes.c_double, _VP, ctypes.c_size_t, _VP, _VP, _VP],
    "wenozn_workspace_status": [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32, _VP],
    "wenozn_last_error": [_VP, ctypes.POINTER(ctypes.c_int32)],
    "wenozn_check_reciprocal": [_VP, ctypes.c_int64, _VP, _VP, _VP],
    "wenozn_fp64_fma_rate": [ctypes.c_int64, ctypes.POINTER(ctypes.c_double), _VP],
    "wenozn_vjp_workspace_size": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "wenozn_rhs_vjp": [_P, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP],
    "wenozn_rk3_step_vjp": [_P, _VP, ctypes.c_double, _VP, _VP, ctypes.c_size_t, _VP],
    "wenozn_rk3_run": [_P, _VP, ctypes.c_int64, ctypes.c_double, _VP, ctypes.c_size_t, _VP],
    "wenozn_rk3_step_keep": [_P, _VP, _VP, ctypes.c_double, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP],
    "wenozn_rk3_run_keep": [_P, _VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_double, _VP, ctypes.c_size_t, _VP],
    "wenozn_rk3_vjp_run": [_P, _VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_double, _VP, _VP, ctypes.c_size_t, _VP],
    "wenozn_rk3_step_vjp_stages": [_P, _VP, _VP, _VP, _VP, ctypes.c_double, _VP, _VP, ctypes.c_size_t, _VP],
    "wenozn_workspace_stages": [_VP, _P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                ctypes.POINTER(ctypes.c_void_p)],
    "wenozn_batch_shape": [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)],
    "wenozn_batch_workspace_size": [ctypes.POINTER(wenozn_batch_params), _VP, ctypes.POINTER(ctypes.c_size_t)],
    "wenozn_batch_init": [ctypes.POINTER(wenozn_batch_params), _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP],
    "wenozn_batch_rk3_step": [ctypes.POINTER(wenozn_batch_params), _VP, _VP, _VP, ctypes.c_size_t, _VP],
    "wenozn_batch_tune": [ctypes.POINTER(wenozn_batch_params), _VP, _VP, _VP, ctypes.c_size_t, ctypes.c_int32,
                          ctypes.POINTER(ctypes.c_float), _VP],
    "wenozn_batch_resolved_shape": [ctypes.POINTER(wenozn_batch_params), _VP, ctypes.POINTER(ctypes.c_int32)],
    "wenozn_batch_state": [_VP, ctypes.c_int32, _VP, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                           ctypes.POINTER(ctypes.c_void_p)],
}


def lib():
    """Load libwenozn.so (raises if it is absent: build it with build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built "
                                   "(python -m paper_2004_07954_gb300.build) - there is no fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.wenozn_status_string.argtypes = [ctypes.c_int]
            L.wenozn_status_string.restype = ctypes.c_char_p
            L.wenozn_version.argtypes = []
            L.wenozn_version.restype = ctypes.c_char_p
            L.wenozn_batch_num_shapes.argtypes = []
            L.wenozn_batch_num_shapes.restype = ctypes.c_int32
            L.wenozn_workspace_dt.argtypes = [_VP]
            L.wenozn_workspace_dt.restype = _VP
            _lib = L
    return _lib


def _check(fn: str, code: int) -> None:
    if code != WENOZN_OK:
        raise WenoznError(fn, code)


def _dev_ptr(t: torch.Tensor, name: str) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


# ------------------------------------------------------------------------- C-ABI mirrors
def wenozn_status_string(code: int) -> str:
    return lib().wenozn_status_string(int(code)).decode()


def wenozn_version() -> str:
    return lib().wenozn_version().decode()


def wenozn_problem_init(system: int, nx: int, ny: int = 1, dx: float = 1.0, dy: float = 1.0,
                        **overrides) -> wenozn_problem:
    p = wenozn_problem()
    _check("wenozn_problem_init", lib().wenozn_problem_init(ctypes.byref(p), int(system), int(nx),
                                                            int(ny), float(dx), float(dy)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def wenozn_workspace_size(p: wenozn_problem) -> int:
    n = ctypes.c_size_t(0)
    _check("wenozn_workspace_size", lib().wenozn_workspace_size(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def workspace(p: wenozn_problem, device=None) -> torch.Tensor:
    """A zero-filled, 256-byte aligned workspace tensor (uint8) for problem p."""
    nbytes = wenozn_workspace_size(p)
    ws = torch.zeros(nbytes + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-ws.data_ptr()) % 256
    return ws[off:off + nbytes]


def wenozn_fill_ghosts(p: wenozn_problem, U_padded: torch.Tensor, stream=None) -> None:
    _check("wenozn_fill_ghosts", lib().wenozn_fill_ghosts(ctypes.byref(p), _dev_ptr(U_padded, "U_padded"),
                                                          _stream(stream)))


def wenozn_reconstruct(f_padded: torch.Tensor, fhat: torch.Tensor, side: int = 1, eps: float = 1e-40,
                       A: float = 10.0, stream=None) -> None:
    n = f_padded.numel() - 6
    if fhat.numel() != n + 1:
        raise ValueError("fhat must hold n + 1 values")
    _check("wenozn_reconstruct", lib().wenozn_reconstruct(_dev_ptr(f_padded, "f_padded"), n,
                                                          _dev_ptr(fhat, "fhat"), int(side), float(eps),
                                                          float(A), _stream(stream)))


def wenozn_reconstruct_weights(f_padded: torch.Tensor, fhat: torch.Tensor, side: int = 1,
                               weights: int = WENOZN_WEIGHTS_ZN, eps: float = 1e-40, A: float = 10.0,
                               stream=None) -> None:
    n = f_padded.numel() - 6
    if fhat.numel() != n + 1:
        raise ValueError("fhat must hold n + 1 values")
    _check("wenozn_reconstruct_weights", lib().wenozn_reconstruct_weights(
        _dev_ptr(f_padded, "f_padded"), n, _dev_ptr(fhat, "fhat"), int(side), int(weights), float(eps),
        float(A), _stream(stream)))


def wenozn_max_wavespeed(p: wenozn_problem, U: torch.Tensor, alpha_out: torch.Tensor,
                         status_dev: torch.Tensor | None = None, stream=None) -> None:
    if alpha_out.numel() < 2:
        raise ValueError("alpha_out must hold 2 values")
    st = 0
    if status_dev is not None:
        if not status_dev.is_cuda or status_dev.dtype != torch.int32:
            raise ValueError("status_dev: expected an int32 CUDA tensor")
        st = status_dev.data_ptr()
    _check("wenozn_max_wavespeed", lib().wenozn_max_wavespeed(ctypes.byref(p), _dev_ptr(U, "U"),
                                                              _dev_ptr(alpha_out, "alpha_out"), st,
                                                              _stream(stream)))


def wenozn_flux(p: wenozn_problem, U: torch.Tensor, alpha: torch.Tensor | None, direction: int,
                Fout: torch.Tensor, stream=None) -> None:
    a = 0 if alpha is None else _dev_ptr(alpha, "alpha")
    _check("wenozn_flux", lib().wenozn_flux(ctypes.byref(p), _dev_ptr(U, "U"), a, int(direction),
                                            _dev_ptr(Fout, "Fout"), _stream(stream)))


def flux_shape(p: wenozn_problem, direction: int):
    """Shape of wenozn_flux's output: one direction's planes, or (direction 2) the x fluxes
    followed by the y fluxes as one flat array."""
    if direction == 2:
        return (p.nvar * (p.ny * (p.nx + 1) + (p.ny + 1) * p.nx),)
    return (p.nvar, p.ny, p.nx + 1) if direction == 0 else (p.nvar, p.ny + 1, p.nx)


def _ws_ptr(ws: torch.Tensor) -> int:
    if not isinstance(ws, torch.Tensor) or not ws.is_cuda:
        raise ValueError("ws: expected a CUDA tensor")
    return ws.data_ptr()


def wenozn_rhs(p: wenozn_problem, U: torch.Tensor, L: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    _check("wenozn_rhs", lib().wenozn_rhs(ctypes.byref(p), _dev_ptr(U, "U"), _dev_ptr(L, "L"), _ws_ptr(ws),
                                          ws.numel() * ws.element_size(), _stream(stream)))


def wenozn_rhs_noalloc(p: wenozn_problem, U: torch.Tensor, L: torch.Tensor, stream=None) -> None:
    """wenozn_rhs with the library's fixed 8 MiB device scratch instead of a workspace, for
    callers that cannot allocate (see the header for limits and sharing rules)."""
    _check("wenozn_rhs_noalloc", lib().wenozn_rhs_noalloc(ctypes.byref(p), _dev_ptr(U, "U"), _dev_ptr(L, "L"),
                                                          _stream(stream)))


def wenozn_rk3_step(p: wenozn_problem, U: torch.Tensor, ws: torch.Tensor, dt: float = 0.0,
                    t_remaining: float = 0.0, return_dt: bool = False, stream=None):
    out = ctypes.c_double(0.0)
    code = lib().wenozn_rk3_step(ctypes.byref(p), _dev_ptr(U, "U"), float(dt), float(t_remaining),
                                 ctypes.byref(out) if return_dt else None, _ws_ptr(ws),
                                 ws.numel() * ws.element_size(), _stream(stream))
    _check("wenozn_rk3_step", code)
    return out.value if return_dt else None


def _host_ptr(t: torch.Tensor, name: str) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float64 host tensor (pinned for asynchronous copies)")
    return t.data_ptr()


def wenozn_rk3_step_host(p: wenozn_problem, U_host_in: torch.Tensor, U_host_out: torch.Tensor,
                         U_dev: torch.Tensor, ws: torch.Tensor, dt: float = 0.0, t_remaining: float = 0.0,
                         return_dt: bool = False, stream=None):
    """One RK3 step of a host-resident state through the device buffer U_dev (copies and
    step enqueued on `stream`)."""
    for t, name in ((U_host_in, "U_host_in"), (U_host_out, "U_host_out"), (U_dev, "U_dev")):
        if t.numel() != p.nvar * p.nx * p.ny:
            raise ValueError(f"{name}: expected {p.nvar * p.nx * p.ny} values")
    out = ctypes.c_double(0.0)
    code = lib().wenozn_rk3_step_host(ctypes.byref(p), _host_ptr(U_host_in, "U_host_in"),
                                      _host_ptr(U_host_out, "U_host_out"), _dev_ptr(U_dev, "U_dev"), float(dt),
                                      float(t_remaining), ctypes.byref(out) if return_dt else None, _ws_ptr(ws),
                                      ws.numel() * ws.element_size(), _stream(stream))
    _check("wenozn_rk3_step_host", code)
    return out.value if return_dt else None


def wenozn_rk3_stream_host(p: wenozn_problem, U_host_in, U_host_out, U_dev0: torch.Tensor, U_dev1: torch.Tensor,
                           ws: torch.Tensor, dt: float = 0.0, stream=None, upload_stream=None,
                           download_stream=None) -> None:
    """One RK3 step of each host state U_host_in[k] into U_host_out[k] (lists of host tensors),
    copies on the two copy streams overlapping the steps on `stream`; asynchronous."""
    if len(U_host_in) != len(U_host_out) or not U_host_in:
        raise ValueError("U_host_in and U_host_out must be non-empty lists of the same length")
    n = p.nvar * p.nx * p.ny
    for t in list(U_host_in) + list(U_host_out) + [U_dev0, U_dev1]:
        if t.numel() != n:
            raise ValueError(f"expected {n} values per state")
    count = len(U_host_in)
    ins = (ctypes.c_void_p * count)(*[_host_ptr(t, "U_host_in") for t in U_host_in])
    outs = (ctypes.c_void_p * count)(*[_host_ptr(t, "U_host_out") for t in U_host_out])
    up = None if upload_stream is None else _stream(upload_stream)
    down = None if download_stream is None else _stream(download_stream)
    _check("wenozn_rk3_stream_host", lib().wenozn_rk3_stream_host(
        ctypes.byref(p), count, ins, outs, _dev_ptr(U_dev0, "U_dev0"), _dev_ptr(U_dev1, "U_dev1"), float(dt),
        _ws_ptr(ws), ws.numel() * ws.element_size(), _stream(stream), up, down))


def wenozn_cfl_dt(p: wenozn_problem, U: torch.Tensor, ws: torch.Tensor, stream=None) -> float:
    """The CFL step of U (the step wenozn_rk3_step would take), computed on the device."""
    out = ctypes.c_double(0.0)
    _check("wenozn_cfl_dt", lib().wenozn_cfl_dt(ctypes.byref(p), _dev_ptr(U, "U"), ctypes.byref(out), _ws_ptr(ws),
                                                ws.numel() * ws.element_size(), _stream(stream)))
    return out.value


def wenozn_last_error(stream=None) -> int:
    """Device status bits raised by the most recent stepping call on `stream` (cleared)."""
    st = ctypes.c_int32(0)
    _check("wenozn_last_error", lib().wenozn_last_error(_stream(stream), ctypes.byref(st)))
    return st.value


def wenozn_workspace_status(ws: torch.Tensor, clear: bool = False, stream=None) -> int:
    st = ctypes.c_int32(0)
    _check("wenozn_workspace_status", lib().wenozn_workspace_status(_ws_ptr(ws), ctypes.byref(st),
                                                                    int(bool(clear)), _stream(stream)))
    return st.value


def wenozn_check_reciprocal(d: torch.Tensor, stream=None):
    """(fast, ieee): the reconstruction's Newton reciprocal and CUDA's IEEE 1/d."""
    fast, ieee = torch.empty_like(d), torch.empty_like(d)
    _check("wenozn_check_reciprocal", lib().wenozn_check_reciprocal(_dev_ptr(d, "d"), d.numel(),
                                                                    _dev_ptr(fast, "fast"), _dev_ptr(ieee, "ieee"),
                                                                    _stream(stream)))
    return fast, ieee


def wenozn_fp64_fma_rate(fmas_per_thread: int = 1 << 17, stream=None) -> float:
    """GFLOP/s of pure FP64 FMA register arithmetic on this GPU (synchronizes the stream)."""
    g = ctypes.c_double(0.0)
    _check("wenozn_fp64_fma_rate", lib().wenozn_fp64_fma_rate(int(fmas_per_thread), ctypes.byref(g), _stream(stream)))
    return g.value


def wenozn_workspace_dt(ws: torch.Tensor) -> torch.Tensor:
    """The device scalar holding the last step taken (a view into the workspace)."""
    addr = lib().wenozn_workspace_dt(_ws_ptr(ws))
    off = addr - ws.data_ptr()
    return ws[off:off + 8].view(torch.float64)


def wenozn_vjp_workspace_size(p: wenozn_problem) -> int:
    n = ctypes.c_size_t(0)
    _check("wenozn_vjp_workspace_size", lib().wenozn_vjp_workspace_size(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def vjp_workspace(p: wenozn_problem, device=None) -> torch.Tensor:
    """Zero-filled, 256-byte aligned workspace for the adjoint (and forward) entry points."""
    nbytes = wenozn_vjp_workspace_size(p)
    ws = torch.zeros(nbytes + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-ws.data_ptr()) % 256
    return ws[off:off + nbytes]


def wenozn_rhs_vjp(p: wenozn_problem, U: torch.Tensor, lam: torch.Tensor, out: torch.Tensor, ws: torch.Tensor,
                   stream=None) -> None:
    _check("wenozn_rhs_vjp", lib().wenozn_rhs_vjp(ctypes.byref(p), _dev_ptr(U, "U"), _dev_ptr(lam, "lam"),
                                                  _dev_ptr(out, "out"), _ws_ptr(ws), ws.numel(), _stream(stream)))


def wenozn_rk3_step_vjp(p: wenozn_problem, U: torch.Tensor, dt: float, lam: torch.Tensor, ws: torch.Tensor,
                        stream=None) -> None:
    _check("wenozn_rk3_step_vjp", lib().wenozn_rk3_step_vjp(ctypes.byref(p), _dev_ptr(U, "U"), float(dt),
                                                            _dev_ptr(lam, "lam"), _ws_ptr(ws), ws.numel(),
                                                            _stream(stream)))


def wenozn_rk3_run(p: wenozn_problem, U: torch.Tensor, nsteps: int, ws: torch.Tensor, dt: float = 0.0,
                   stream=None) -> None:
    _check("wenozn_rk3_run", lib().wenozn_rk3_run(ctypes.byref(p), _dev_ptr(U, "U"), int(nsteps), float(dt),
                                                  _ws_ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def wenozn_rk3_step_keep(p: wenozn_problem, U: torch.Tensor, U_next: torch.Tensor, dt: float, U1: torch.Tensor,
                         U2: torch.Tensor, alphas: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    _check("wenozn_rk3_step_keep", lib().wenozn_rk3_step_keep(
        ctypes.byref(p), _dev_ptr(U, "U"), _dev_ptr(U_next, "U_next"), float(dt), _dev_ptr(U1, "U1"),
        _dev_ptr(U2, "U2"), _dev_ptr(alphas, "alphas"), _ws_ptr(ws), ws.numel() * ws.element_size(),
        _stream(stream)))


def wenozn_rk3_run_keep(p: wenozn_problem, X: torch.Tensor, S1: torch.Tensor, S2: torch.Tensor,
                        alphas: torch.Tensor, nsteps: int, dt: float, ws: torch.Tensor, stream=None) -> None:
    _check("wenozn_rk3_run_keep", lib().wenozn_rk3_run_keep(
        ctypes.byref(p), _dev_ptr(X, "X"), _dev_ptr(S1, "S1"), _dev_ptr(S2, "S2"), _dev_ptr(alphas, "alphas"),
        int(nsteps), float(dt), _ws_ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def wenozn_rk3_vjp_run(p: wenozn_problem, X: torch.Tensor, S1: torch.Tensor, S2: torch.Tensor,
                       alphas: torch.Tensor, nsteps: int, dt: float, lam: torch.Tensor, ws: torch.Tensor,
                       stream=None) -> None:
    _check("wenozn_rk3_vjp_run", lib().wenozn_rk3_vjp_run(
        ctypes.byref(p), _dev_ptr(X, "X"), _dev_ptr(S1, "S1"), _dev_ptr(S2, "S2"), _dev_ptr(alphas, "alphas"),
        int(nsteps), float(dt), _dev_ptr(lam, "lam"), _ws_ptr(ws), ws.numel() * ws.element_size(),
        _stream(stream)))


def wenozn_rk3_step_vjp_stages(p: wenozn_problem, U: torch.Tensor, U1: torch.Tensor, U2: torch.Tensor,
                               alphas: torch.Tensor, dt: float, lam: torch.Tensor, ws: torch.Tensor,
                               stream=None) -> None:
    _check("wenozn_rk3_step_vjp_stages", lib().wenozn_rk3_step_vjp_stages(
        ctypes.byref(p), _dev_ptr(U, "U"), _dev_ptr(U1, "U1"), _dev_ptr(U2, "U2"), _dev_ptr(alphas, "alphas"),
        float(dt), _dev_ptr(lam, "lam"), _ws_ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def workspace_stages(p: wenozn_problem, ws: torch.Tensor):
    """Views (U1, U2, alphas[3]) of the last forward RK3 step's stage inputs and LF speeds."""
    u1, u2, al = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check("wenozn_workspace_stages", lib().wenozn_workspace_stages(_ws_ptr(ws), ctypes.byref(p), ctypes.byref(u1),
                                                                    ctypes.byref(u2), ctypes.byref(al)))
    nb = p.nvar * p.nx * p.ny * 8
    base = ws.data_ptr()
    U1 = ws[u1.value - base:u1.value - base + nb].view(torch.float64).view(p.shape)
    U2 = ws[u2.value - base:u2.value - base + nb].view(torch.float64).view(p.shape)
    A = ws[al.value - base:al.value - base + 48].view(torch.float64)[0::2]
    return U1, U2, A


# ------------------------------------------------------------------------- convenience
class Solver:
    """One problem, one workspace: RHS evaluations and RK3 steps on torch tensors."""

    def __init__(self, p: wenozn_problem, device=None):
        self.p = p
        self.ws = workspace(p, device)

    def rhs(self, U: torch.Tensor, L: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if L is None:
            L = torch.empty_like(U)
        wenozn_rhs(self.p, U, L, self.ws, stream)
        return L

    def step(self, U: torch.Tensor, dt: float = 0.0, t_remaining: float = 0.0, return_dt=False, stream=None):
        return wenozn_rk3_step(self.p, U, self.ws, dt, t_remaining, return_dt, stream)

    def steps(self, U: torch.Tensor, n: int, dt: float = 0.0, stream=None) -> None:
        """n RK3 steps in one asynchronous call (no clipping at a final time)."""
        wenozn_rk3_run(self.p, U, n, self.ws, dt, stream)

    def run(self, U: torch.Tensor, T: float, dt: float = 0.0, stream=None) -> int:
        """Advance to time T (CFL steps clipped at T, or fixed steps); returns steps."""
        if dt > 0:
            import math
            n = int(math.ceil(T / dt - 1e-9))
            for k in range(n):
                self.step(U, dt=(T - k * dt) if k == n - 1 else dt, stream=stream)
            return n
        t, steps = 0.0, 0
        while t < T * (1 - 1e-14):
            t += self.step(U, t_remaining=T - t, return_dt=True, stream=stream)
            steps += 1
        return steps

    def status(self, clear: bool = False) -> int:
        return wenozn_workspace_status(self.ws, clear)


# ------------------------------------------------------------------------- batched 1D Euler
def wenozn_batch_num_shapes() -> int:
    return lib().wenozn_batch_num_shapes()


def wenozn_batch_shape(shape: int):
    t, th = ctypes.c_int32(0), ctypes.c_int32(0)
    _check("wenozn_batch_shape", lib().wenozn_batch_shape(int(shape), ctypes.byref(t), ctypes.byref(th)))
    return t.value, th.value


class Batch:
    """B independent 1D Euler problems in one concatenated state U[3][total] (float64, CUDA),
    instance b at columns offsets[b]:offsets[b+1] with spacing dx[b]."""

    def __init__(self, offsets, dx, U: torch.Tensor, *, bc=WENOZN_BC_OUTFLOW, shape=-1, t_final=0.0,
                 gamma=1.4, eps=1e-40, A=10.0, cfl=0.5, device=None):
        import numpy as np
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.dx = np.ascontiguousarray(dx, dtype=np.float64)
        B = self.offsets.size - 1
        if self.dx.size != B:
            raise ValueError("dx must hold one spacing per instance")
        self.bp = wenozn_batch_params(B, bc, shape, 0, gamma, eps, A, cfl, t_final)
        n = ctypes.c_size_t(0)
        _check("wenozn_batch_workspace_size", lib().wenozn_batch_workspace_size(
            ctypes.byref(self.bp), self.offsets.ctypes.data, ctypes.byref(n)))
        ws = torch.zeros(n.value + 256, dtype=torch.uint8, device=device or U.device)
        off = (-ws.data_ptr()) % 256
        self.ws = ws[off:off + n.value]
        self.init(U)

    @property
    def nbatch(self) -> int:
        return self.bp.nbatch

    def init(self, U: torch.Tensor, stream=None) -> None:
        _check("wenozn_batch_init", lib().wenozn_batch_init(
            ctypes.byref(self.bp), self.offsets.ctypes.data, self.dx.ctypes.data, _dev_ptr(U, "U"),
            self.ws.data_ptr(), self.ws.numel(), _stream(stream)))

    def step(self, U: torch.Tensor, stream=None) -> None:
        _check("wenozn_batch_rk3_step", lib().wenozn_batch_rk3_step(
            ctypes.byref(self.bp), self.offsets.ctypes.data, _dev_ptr(U, "U"), self.ws.data_ptr(),
            self.ws.numel(), _stream(stream)))

    def shape_in_use(self) -> int:
        """The tile shape a step of this batch uses (its own, the tuning table's or the default)."""
        sh = ctypes.c_int32(0)
        _check("wenozn_batch_resolved_shape", lib().wenozn_batch_resolved_shape(
            ctypes.byref(self.bp), self.offsets.ctypes.data, ctypes.byref(sh)))
        return sh.value

    def tune(self, U_scratch: torch.Tensor, steps: int = 2, stream=None):
        """Times every compiled tile shape on U_scratch (advanced by the trials) and keeps the
        fastest, also in the process-wide table of this batch's size class; steps = 0 reuses
        the table's entry without timing when there is one.  Returns the per-shape
        milliseconds per step (zeros when nothing was timed)."""
        ms = (ctypes.c_float * wenozn_batch_num_shapes())()
        _check("wenozn_batch_tune", lib().wenozn_batch_tune(
            ctypes.byref(self.bp), self.offsets.ctypes.data, _dev_ptr(U_scratch, "U"), self.ws.data_ptr(),
            self.ws.numel(), int(steps), ms, _stream(stream)))
        return list(ms)

    def _state_ptrs(self):
        t, dt, st = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check("wenozn_batch_state", lib().wenozn_batch_state(self.ws.data_ptr(), self.nbatch,
                                                              self.offsets.ctypes.data, ctypes.byref(t),
                                                              ctypes.byref(dt), ctypes.byref(st)))
        return t.value, dt.value, st.value

    def _view(self, addr: int, count: int, dtype) -> torch.Tensor:
        off = addr - self.ws.data_ptr()
        return self.ws[off:off + count * torch.empty((), dtype=dtype).element_size()].view(dtype)

    def times(self) -> torch.Tensor:
        return self._view(self._state_ptrs()[0], self.nbatch, torch.float64)

    def steps_taken(self) -> torch.Tensor:
        return self._view(self._state_ptrs()[1], self.nbatch, torch.float64)

    def status(self) -> int:
        torch.cuda.synchronize()
        return int(self._view(self._state_ptrs()[2], 1, torch.int32).item())

    def capture(self, U: torch.Tensor, steps: int) -> "torch.cuda.CUDAGraph":
        """A CUDA graph of `steps` RK3 steps of the batch on U (replay with .replay())."""
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            for _ in range(steps):
                self.step(U)
        return g
