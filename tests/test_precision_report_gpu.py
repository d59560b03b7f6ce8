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
