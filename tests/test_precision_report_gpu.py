"""Error against the FP64 oracle per storage format (the precision sweep's
formats): a 256 x 512 crop of the 3840x2160 piecewise-smooth scene, stored
as uint8, FP16, BF16 and FP32 (float formats hold u8/255), zoomed with FP32
arithmetic, compared with the oracle run on the values each format actually
holds, and with the oracle run on the scene values themselves (u8/255, so
that the format's own input rounding is included).  Prints max and mean
|error| in units of the pixel range [0, 1]."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2312_00229_gb300 import api, scenes

pytestmark = pytest.mark.gpu

BOUNDS = {  # max |error| allowed (pixel range 1): the parity tolerances
    "u8": 0.5 / 255 + 1e-5, "f16": 2 ** -11 + 1e-5, "bf16": 2 ** -8 + 1e-5, "f32": 1e-5}


def test_error_per_storage_format():
    img = scenes.piecewise_smooth(2160, 3840, seed=scenes.seed_for(4))
    crop = scenes.planar(img)[:, 960:1216, 1600:2112]
    lines = []
    scene = crop.astype(np.float64) / 255.0
    ref_scene = oracle.zoom2x(scene)
    for dt in ("u8", "f16", "bf16", "f32"):
        x = parity.encode(crop.astype(np.float64) / 255.0, dt)
        held = parity.decode(x)                      # the values the format holds
        ref = oracle.zoom2x(held)
        y = api.zoom2x_fwd(x.cuda())
        torch.cuda.synchronize()
        err = np.abs(parity.decode(y) - (np.clip(ref, 0, 1) if dt == "u8" else ref))
        e2 = np.abs(parity.decode(y) - (np.clip(ref_scene, 0, 1) if dt == "u8" else ref_scene))
        lines.append(f"{dt}: max {err.max():.3e} mean {err.mean():.3e} (vs the scene values: "
                     f"max {e2.max():.3e} mean {e2.mean():.3e})")
        assert err.max() <= BOUNDS[dt], lines[-1]
    print("\nerror vs FP64 oracle (pixel range 1): " + "; ".join(lines))


def test_cascade8x_error_per_storage_format():
    """The precision sweep's 8x cascade (three 2x levels, h halving per level,
    FP32 between levels) on a 64 x 80 crop of the 512 x 512 pixel-art frame,
    stored and returned in each format, against the FP64 oracle run three
    times on the values the format holds, with no rounding between levels.
    Allowed: the output format's half unit plus one FP32 tolerance per level;
    uint8 codes off by one only within three tie windows of a .5 boundary."""
    img = scenes.pixel_art(512, 512, seed=scenes.seed_for(4, 1))
    crop = scenes.planar(img)[:, 200:264, 100:180]
    tol32 = 3 * parity.F32_TOL
    lines = []
    for dt in ("u8", "f16", "bf16", "f32"):
        x = parity.encode(crop.astype(np.float64) / 255.0, dt)
        ref = parity.decode(x)
        for lvl in range(3):
            ref = oracle.zoom2x(ref, h=1.0 / (1 << lvl))
        y = api.cascade_zoom(x.cuda(), 3)
        torch.cuda.synchronize()
        assert y.dtype == x.dtype and y.shape == (3, 512, 640)
        g = parity.decode(y)
        if dt == "u8":
            r = np.clip(ref, 0.0, 1.0)
            diff = y.cpu().numpy().astype(np.int64) - oracle.encode_u8(ref).astype(np.int64)
            scaled = r * 255.0
            near_tie = np.abs(scaled - np.floor(scaled) - 0.5) <= 3 * parity.TIE_WINDOW
            assert np.abs(diff).max() <= 1 and np.all(near_tie[diff != 0])
            err = np.abs(g - r)
            lines.append(f"{dt}: max {err.max():.3e} mean {err.mean():.3e} "
                         f"({int((diff != 0).sum())} tie codes)")
        else:
            err = np.abs(g - ref)
            tol = tol32 + (0.5 * parity.ulp(ref, dt) if dt != "f32" else 0.0)
            assert np.all(err <= tol), f"{dt}: worst excess {(err - tol).max():.3g}"
            lines.append(f"{dt}: max {err.max():.3e} mean {err.mean():.3e}")
    print("\n8x cascade error vs FP64 oracle (pixel range 1): " + "; ".join(lines))
