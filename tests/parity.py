"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64
oracle on the same decoded inputs and compare with the stated tolerances.

Tolerances (derivation in the design notes):
  * FP32 outputs: max |gpu - oracle| <= 1e-5 x (pixel range of the input).
  * uint8 outputs: identical to the oracle's round-half-even encoding, except
    for off-by-one codes whose FP64 value sits within 255 x 1e-5 of a .5
    rounding boundary (ties decided by FP32 vs FP64 rounding); the count of
    such ties is returned so tests can report it.
  * FP16 / BF16 outputs: |gpu - oracle| <= half an ulp of the storage format
    at the oracle value, plus the FP32 tolerance.
"""
import numpy as np
import torch

import oracle
from paper_2312_00229_gb300 import api

F32_TOL = 1e-5
TIE_WINDOW = 255.0 * F32_TOL

TORCH_DT = {"u8": torch.uint8, "f16": torch.float16, "bf16": torch.bfloat16,
            "f32": torch.float32}


def decode(arr_t: torch.Tensor) -> np.ndarray:
    """Storage -> float64 values the method sees (uint8 is v / 255)."""
    a = arr_t.detach().cpu()
    if a.dtype == torch.uint8:
        return a.numpy().astype(np.float64) / 255.0
    return a.to(torch.float64).numpy()


def encode(x: np.ndarray, dt: str) -> torch.Tensor:
    """float values in [0, 1] -> storage tensor (CPU)."""
    if dt == "u8":
        return torch.from_numpy(np.rint(np.clip(x, 0, 1) * 255.0).astype(np.uint8))
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(TORCH_DT[dt])


def oracle_planes(A: np.ndarray, params: api.Params) -> np.ndarray:
    """Oracle on [..., H, W] planes."""
    return oracle.zoom2x(A, beta=params.beta, k_eps=params.k_eps, h=params.h,
                         nbr_c=(params.nbr_c, params.nbr_c),
                         si_scale=params.si_scale, out_mode=params.out_mode)


def ulp(v: np.ndarray, dt: str) -> np.ndarray:
    a = np.abs(v)
    if dt == "f16":
        return np.spacing(a.astype(np.float16)).astype(np.float64)
    # bfloat16: 8 significant bits, FP32 exponent range
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -126)))
    return 2.0 ** (e - 7)


def compare(gpu_out: torch.Tensor, ref: np.ndarray, dt: str, value_range: float = 1.0,
            clamp_float: bool = False):
    """Asserts the tolerance for storage type `dt`; returns (max_err, ties)."""
    g = decode(gpu_out)
    assert g.shape == ref.shape, (g.shape, ref.shape)
    if dt == "u8":
        want = oracle.encode_u8(ref)
        diff = gpu_out.cpu().numpy().astype(np.int64) - want.astype(np.int64)
        bad = np.abs(diff) > 1
        assert not bad.any(), f"{bad.sum()} uint8 codes off by more than one"
        scaled = np.clip(ref, 0.0, 1.0) * 255.0
        near_tie = np.abs(scaled - np.floor(scaled) - 0.5) <= TIE_WINDOW
        off = diff != 0
        assert np.all(near_tie[off]), (
            f"{int((off & ~near_tie).sum())} off-by-one codes are not rounding ties")
        return float(np.abs(g - np.clip(ref, 0, 1)).max()), int(off.sum())
    r = np.clip(ref, 0.0, 1.0) if clamp_float else ref
    err = np.abs(g - r)
    tol = F32_TOL * value_range
    if dt in ("f16", "bf16"):
        tol = tol + 0.5 * ulp(r, dt)
    assert np.all(err <= tol), f"max err {err.max():.3g} (worst excess {(err - tol).max():.3g})"
    return float(err.max()), 0
