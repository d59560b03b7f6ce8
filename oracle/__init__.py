"""FP64 CPU oracle for the WD WENO 2x zoom (arXiv 2312.00229, Sec. 3).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The CUDA library in
``paper_2312_00229_gb300`` never imports it, and it imports nothing from there.

Two independent restatements live here:

* ``wdweno_oracle.c`` (compiled to ``_build/liboracle.so``): the method written
  as plain double-precision loops over a fine-grid array, in the order of
  Algorithms 1 and 2.  ``zoom2x`` below calls it.
* ``wdweno_torch.py``: a vectorised float64 PyTorch restatement used where a
  gradient is needed (autograd gives the FP64 reference gradient).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "wdweno_oracle.c"), os.path.join(_HERE, "wenospline_oracle.c")]

SI_NORMALIZED, SI_LITERAL = 0, 1
OUT_2N, OUT_2N_MINUS_1 = 0, 1
BC_CLAMP, BC_ZERO, BC_REFLECT101, BC_SYMMETRIC = 0, 1, 2, 3


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("beta", ctypes.c_double),
        ("k_eps", ctypes.c_double),
        ("h", ctypes.c_double),
        ("si_scale", ctypes.c_int),
        ("out_mode", ctypes.c_int),
        ("boundary", ctypes.c_int),
        ("ghost", ctypes.c_int),
        ("nbr_c1", ctypes.c_double),
        ("nbr_c2", ctypes.c_double),
    ]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain C99, -O2, OpenMP across planes)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [s for s in _SOURCES if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "wdweno_oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.oracle_params_default.restype = OracleParams
            L.oracle_zoom2x.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.POINTER(OracleParams)]
            L.oracle_zoom2x_planes.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_void_p,
                                               ctypes.POINTER(OracleParams)]
            L.oracle_zoom2x_banded.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_int64, ctypes.c_void_p,
                                               ctypes.POINTER(OracleParams), ctypes.c_int64,
                                               ctypes.c_int]
            L.oracle_encode_u8.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
            L.oracle_encode_u8.restype = None
            L.oracle_directional.argtypes = [ctypes.c_double] * 4 + [
                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.oracle_directional.restype = None
            L.oracle_weno1d_cell.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.oracle_weno1d_cell.restype = ctypes.c_double
            L.oracle_weno_spline.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double]
            L.oracle_weno_spline.restype = ctypes.c_double
            L.oracle_tensor_resample.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                 ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double]
            _lib = L
    return _lib


def params(beta=2.0, k_eps=1e-8, h=1.0, si_scale=SI_NORMALIZED, out_mode=OUT_2N,
           boundary=BC_CLAMP, ghost=None, nbr_c=None) -> OracleParams:
    """`nbr_c` = (phase-1, phase-2) coefficients c of the neighbour weight
    c h^2 in D (Eqs. 2DsmoothnessFinal, tezine); None keeps the default."""
    p = lib().oracle_params_default()
    p.beta, p.k_eps, p.h = float(beta), float(k_eps), float(h)
    p.si_scale, p.out_mode, p.boundary = int(si_scale), int(out_mode), int(boundary)
    if ghost is not None:
        p.ghost = int(ghost)
    if nbr_c is not None:
        p.nbr_c1, p.nbr_c2 = float(nbr_c[0]), float(nbr_c[1])
    return p


def out_shape(n: int, m: int, out_mode: int = OUT_2N):
    return (2 * n - 1, 2 * m - 1) if out_mode == OUT_2N_MINUS_1 else (2 * n, 2 * m)


def zoom2x(A, beta=2.0, k_eps=1e-8, h=1.0, si_scale=SI_NORMALIZED, out_mode=OUT_2N,
           boundary=BC_CLAMP, ghost=None, nbr_c=None) -> np.ndarray:
    """WD WENO 2x zoom of ``A`` (shape [..., n, m]) in float64.

    Leading dimensions are independent planes (channels, images)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    if A.ndim < 2:
        raise ValueError("need at least 2 dimensions")
    lead = A.shape[:-2]
    n, m = A.shape[-2:]
    planes = int(np.prod(lead)) if lead else 1
    orows, ocols = out_shape(n, m, out_mode)
    U = np.empty(lead + (orows, ocols), dtype=np.float64)
    prm = params(beta, k_eps, h, si_scale, out_mode, boundary, ghost, nbr_c)
    rc = lib().oracle_zoom2x_planes(A.ctypes.data, planes, n, m, U.ctypes.data, ctypes.byref(prm))
    if rc != 0:
        raise RuntimeError(f"oracle_zoom2x failed with code {rc}")
    return U


def zoom2x_banded(A, band_rows=16, threads=0, beta=2.0, k_eps=1e-8, h=1.0,
                  si_scale=SI_NORMALIZED, out_mode=OUT_2N, nbr_c=None) -> np.ndarray:
    """``zoom2x`` computed in row bands on `threads` host threads (0 = all
    OpenMP threads).  Same values; used to time the oracle on many cores."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    lead = A.shape[:-2]
    n, m = A.shape[-2:]
    planes = int(np.prod(lead)) if lead else 1
    orows, ocols = out_shape(n, m, out_mode)
    U = np.empty(lead + (orows, ocols), dtype=np.float64)
    prm = params(beta, k_eps, h, si_scale, out_mode, BC_CLAMP, None, nbr_c)
    rc = lib().oracle_zoom2x_banded(A.ctypes.data, planes, n, m, U.ctypes.data,
                                    ctypes.byref(prm), int(band_rows), int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_zoom2x_banded failed with code {rc}")
    return U


def directional(n0, n1, n2, scale_over_step=2.0):
    """(p, SI) of one stencil, nodes at t = -1, 1, 3 fine steps."""
    p, si = ctypes.c_double(), ctypes.c_double()
    lib().oracle_directional(float(n0), float(n1), float(n2), float(scale_over_step),
                             ctypes.byref(p), ctypes.byref(si))
    return p.value, si.value


def encode_u8(U) -> np.ndarray:
    """Saturate to [0, 1], scale by 255, round half to even (float64 decision)."""
    U = np.ascontiguousarray(np.asarray(U, dtype=np.float64))
    out = np.empty(U.shape, dtype=np.uint8)
    lib().oracle_encode_u8(U.ctypes.data, U.size, out.ctypes.data)
    return out


def weno1d_cell(v4, t, beta=2.0, k_eps=1e-8, h=1.0) -> float:
    """1-D WENO interpolant of Sec. 2 on the cell [x_i, x_{i+1}] (t in [0, 1])."""
    arr = (ctypes.c_double * 4)(*[float(v) for v in v4])
    return lib().oracle_weno1d_cell(arr, float(t), float(beta), float(k_eps), float(h))


def weno_spline(V, x, beta=2.0, k_eps=1e-8, h=1.0) -> float:
    """WENO spline w(V, x) of Sec. 3.3 on the grid 0..n-1 (clamped ends)."""
    V = np.ascontiguousarray(np.asarray(V, dtype=np.float64))
    return lib().oracle_weno_spline(V.ctypes.data, V.size, 1, float(x), float(beta),
                                    float(k_eps), float(h))


def tensor_resample(A, out_h, out_w, beta=2.0, k_eps=1e-8, h=1.0) -> np.ndarray:
    """Eq. (tensor): resample [..., n, m] planes to out_h x out_w on the
    endpoint-aligned grids."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    lead = A.shape[:-2]
    n, m = A.shape[-2:]
    planes = A.reshape(-1, n, m)
    U = np.empty((planes.shape[0], out_h, out_w), dtype=np.float64)
    for p in range(planes.shape[0]):
        src = np.ascontiguousarray(planes[p])
        rc = lib().oracle_tensor_resample(src.ctypes.data, n, m, U[p].ctypes.data, out_h, out_w,
                                          float(beta), float(k_eps), float(h))
        if rc != 0:
            raise RuntimeError(f"oracle_tensor_resample failed with code {rc}")
    return U.reshape(lead + (out_h, out_w))


def zoom_to(A, out_h, out_w, beta=2.0, k_eps=1e-8, h=1.0) -> np.ndarray:
    """Arbitrary-resolution zoom of Sec. 3.3: k successive WD WENO doublings
    on the (2n-1) grid (Eq. zoomfactor) up to the first size >= the target in
    both directions, then tensor WENO resampling to out_h x out_w.  Each
    level's coarse spacing is half the previous level's."""
    A = np.asarray(A, dtype=np.float64)
    cur, hc = A, float(h)
    while ((cur.shape[-2] < out_h and cur.shape[-2] > 1)
           or (cur.shape[-1] < out_w and cur.shape[-1] > 1)):
        cur = zoom2x(cur, beta=beta, k_eps=k_eps, h=hc, out_mode=OUT_2N_MINUS_1)
        hc = hc / 2.0
    return tensor_resample(cur, out_h, out_w, beta=beta, k_eps=k_eps, h=hc)
