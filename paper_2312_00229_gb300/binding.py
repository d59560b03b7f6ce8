"""ctypes binding of ``libwdweno.so`` (C ABI: ``include/wdweno.h``).

Argument marshalling only: every function here forwards to the CUDA library
under the same name.  Loading fails loudly when the library is missing; there
is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

WENO_OK, WENO_EINVAL, WENO_EDTYPE, WENO_EWORKSPACE, WENO_ECUDA, WENO_ERANGE = 0, -1, -2, -3, -4, -5
WENO_U8, WENO_F16, WENO_BF16, WENO_F32 = 0, 1, 2, 3
WENO_OUT_2N, WENO_OUT_2N_MINUS_1 = 0, 1
WENO_SI_NORMALIZED, WENO_SI_LITERAL_SQRT2H = 0, 1

# Every exported symbol of include/wdweno.h.
EXPORTS = (
    "weno_params_default",
    "weno_status_string",
    "weno_zoom2x_fwd",
    "weno_zoom2x_fwd_tiled",
    "weno_zoom2x_bwd",
    "weno_zoom2x_bwd_workspace_bytes",
    "weno_zoom2x_batched_workspace_bytes",
    "weno_zoom2x_batched",
    "weno_zoom2x_batched_noalloc",
    "weno_resample",
    "weno_zoom2x_cascade",
    "weno_zoom2x_cascade_workspace_bytes",
    "weno_wait_timeouts",
    "weno_fp32_probe",
    "weno_fp32_probe_ops",
)
WENO_NOALLOC_MAX_IMAGES = 4096
WENO_CASCADE_MAX_LEVELS = 6


class weno_params(ctypes.Structure):
    _fields_ = [
        ("beta", ctypes.c_float),
        ("k_eps", ctypes.c_float),
        ("h", ctypes.c_float),
        ("si_scale", ctypes.c_int),
        ("out_mode", ctypes.c_int),
        ("clamp_float", ctypes.c_int),
        ("data_bound", ctypes.c_float),
        ("nbr_c", ctypes.c_float),
    ]


class weno_image(ctypes.Structure):
    _fields_ = [
        ("data", ctypes.c_void_p),
        ("height", ctypes.c_int64),
        ("width", ctypes.c_int64),
        ("channels", ctypes.c_int64),
        ("stride_c", ctypes.c_int64),
        ("stride_h", ctypes.c_int64),
        ("stride_w", ctypes.c_int64),
    ]


_P = ctypes.POINTER
_IMG = _P(weno_image)
_PRM = _P(weno_params)
_VP = ctypes.c_void_p

_SIGS = {
    "weno_params_default": ([], weno_params),
    "weno_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "weno_zoom2x_fwd": ([_IMG, ctypes.c_int, _IMG, ctypes.c_int, _PRM, _VP], ctypes.c_int),
    "weno_zoom2x_fwd_tiled": ([_IMG, ctypes.c_int, _IMG, ctypes.c_int, _PRM, ctypes.c_int,
                               ctypes.c_int, _VP], ctypes.c_int),
    "weno_zoom2x_bwd": ([_IMG, _IMG, _IMG, _PRM, _VP, ctypes.c_size_t, _VP], ctypes.c_int),
    "weno_zoom2x_bwd_workspace_bytes": ([_IMG], ctypes.c_size_t),
    "weno_zoom2x_batched_workspace_bytes": ([ctypes.c_int], ctypes.c_size_t),
    "weno_zoom2x_batched": ([ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _PRM, _VP,
                             ctypes.c_size_t, ctypes.c_int, ctypes.c_int, _VP], ctypes.c_int),
    "weno_zoom2x_batched_noalloc": ([ctypes.c_int, _VP, ctypes.c_int, _VP, ctypes.c_int, _PRM,
                                     ctypes.c_int, ctypes.c_int, _VP], ctypes.c_int),
    "weno_resample": ([_IMG, ctypes.c_int, _IMG, ctypes.c_int, _PRM, _VP], ctypes.c_int),
    "weno_wait_timeouts": ([ctypes.POINTER(ctypes.c_uint), ctypes.c_int], ctypes.c_int),
    "weno_zoom2x_cascade": ([_IMG, ctypes.c_int, _IMG, ctypes.c_int, ctypes.c_int, _PRM, _VP,
                             ctypes.c_size_t, _VP], ctypes.c_int),
    "weno_zoom2x_cascade_workspace_bytes": ([_IMG, ctypes.c_int, _PRM], ctypes.c_size_t),
    "weno_fp32_probe": ([ctypes.c_int, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "weno_fp32_probe_ops": ([ctypes.c_int, ctypes.c_int], ctypes.c_longlong),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads (building first if needed) and returns the CDLL."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libwdweno.so not found at {path}")
            L = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


class WenoError(RuntimeError):
    def __init__(self, func: str, status: int):
        msg = load().weno_status_string(status).decode()
        super().__init__(f"{func} failed with status {status}: {msg}")
        self.status = status


def check(func: str, status: int) -> None:
    if status != WENO_OK:
        raise WenoError(func, status)


def weno_params_default() -> weno_params:
    return load().weno_params_default()


def weno_status_string(status: int) -> str:
    return load().weno_status_string(int(status)).decode()


def weno_zoom2x_fwd(inp, in_t, out, out_t, params, stream) -> int:
    return load().weno_zoom2x_fwd(ctypes.byref(inp), in_t, ctypes.byref(out), out_t,
                                  ctypes.byref(params) if params is not None else None, stream)


def weno_zoom2x_fwd_tiled(inp, in_t, out, out_t, params, rows_per_tile, tile_width, stream) -> int:
    return load().weno_zoom2x_fwd_tiled(ctypes.byref(inp), in_t, ctypes.byref(out), out_t,
                                        ctypes.byref(params) if params is not None else None,
                                        int(rows_per_tile), int(tile_width), stream)


def weno_zoom2x_bwd(x, grad_out, grad_in, params, workspace, workspace_bytes, stream) -> int:
    return load().weno_zoom2x_bwd(ctypes.byref(x), ctypes.byref(grad_out), ctypes.byref(grad_in),
                                  ctypes.byref(params) if params is not None else None,
                                  workspace, int(workspace_bytes), stream)


def weno_zoom2x_bwd_workspace_bytes(x) -> int:
    return int(load().weno_zoom2x_bwd_workspace_bytes(ctypes.byref(x)))


def weno_zoom2x_batched_workspace_bytes(count: int) -> int:
    return int(load().weno_zoom2x_batched_workspace_bytes(int(count)))


def weno_zoom2x_batched(count, d_in, in_t, d_out, out_t, params, workspace, workspace_bytes,
                        rows_per_tile, tile_width, stream) -> int:
    return load().weno_zoom2x_batched(int(count), d_in, in_t, d_out, out_t,
                                      ctypes.byref(params) if params is not None else None,
                                      workspace, int(workspace_bytes), int(rows_per_tile),
                                      int(tile_width), stream)


def weno_zoom2x_batched_noalloc(count, d_in, in_t, d_out, out_t, params, rows_per_tile,
                                tile_width, stream) -> int:
    return load().weno_zoom2x_batched_noalloc(int(count), d_in, in_t, d_out, out_t,
                                              ctypes.byref(params) if params is not None else None,
                                              int(rows_per_tile), int(tile_width), stream)


def weno_resample(inp, in_t, out, out_t, params, stream) -> int:
    return load().weno_resample(ctypes.byref(inp), in_t, ctypes.byref(out), out_t,
                                ctypes.byref(params) if params is not None else None, stream)


def weno_zoom2x_cascade(inp, in_t, out, out_t, levels, params, workspace, workspace_bytes,
                        stream) -> int:
    return load().weno_zoom2x_cascade(ctypes.byref(inp), in_t, ctypes.byref(out), out_t,
                                      int(levels),
                                      ctypes.byref(params) if params is not None else None,
                                      workspace, int(workspace_bytes), stream)


def weno_zoom2x_cascade_workspace_bytes(inp, levels, params) -> int:
    return load().weno_zoom2x_cascade_workspace_bytes(
        ctypes.byref(inp), int(levels), ctypes.byref(params) if params is not None else None)


def weno_wait_timeouts(reset: bool = False) -> int:
    """Abandoned bounded waits of the fused cascade's kernels (raises on error)."""
    v = ctypes.c_uint(0)
    check("weno_wait_timeouts", load().weno_wait_timeouts(ctypes.byref(v), 1 if reset else 0))
    return int(v.value)


def weno_fp32_probe(blocks, iters, out, stream) -> int:
    return load().weno_fp32_probe(int(blocks), int(iters), out, stream)


def weno_fp32_probe_ops(blocks, iters) -> int:
    return int(load().weno_fp32_probe_ops(int(blocks), int(iters)))
