"""Fused 2^k cascade (Sec. 3.3, Eq. zoomfactor): one persistent launch over
every level equals the level-by-level cascade bit for bit (same tile body,
same per-level parameters), and waits between levels never give up."""
import numpy as np
import pytest
import torch

from paper_2312_00229_gb300 import api, binding as B, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _img(h, w, dtype, seed):
    g = torch.Generator(device=DEV).manual_seed(seed)
    t = torch.randint(0, 256, (3, h, w), device=DEV, generator=g, dtype=torch.uint8)
    return t if dtype == torch.uint8 else (t.float() / 255.0).to(dtype)


@pytest.mark.parametrize("dtype", [torch.uint8, torch.float16, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("levels", [1, 2, 3])
def test_fused_equals_level_by_level(dtype, mode, levels):
    x = _img(37, 61, dtype, seed=levels * 10 + mode)
    p = api.Params(out_mode=mode)
    a = api.cascade_zoom(x, levels, p, fused=True)
    b = api.cascade_zoom(x, levels, p)
    torch.cuda.synchronize()
    assert a.shape == b.shape and a.dtype == b.dtype
    assert torch.equal(a, b)


@pytest.mark.parametrize("shape", [(1, 1), (2, 300), (300, 2), (130, 500), (512, 512)])
def test_fused_shapes_and_waits(shape):
    """Bands of consecutive levels straddle each other at every size; no wait
    between levels gives up."""
    B.weno_wait_timeouts(reset=True)
    x = torch.from_numpy(np.ascontiguousarray(scenes.planar(
        scenes.pixel_art(shape[0], shape[1], seed=scenes.seed_for(4, 20))))).to(DEV)
    a = api.cascade_zoom(x, 3, fused=True)
    b = api.cascade_zoom(x, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert B.weno_wait_timeouts() == 0


def test_fused_general_beta_and_params():
    x = _img(45, 70, torch.float32, seed=3)
    for p in (api.Params(beta=1.0), api.Params(beta=0.0), api.Params(h=0.25, k_eps=1e-4),
              api.Params(si_scale=1, data_bound=1.0)):
        a = api.cascade_zoom(x, 2, p, fused=True)
        b = api.cascade_zoom(x, 2, p)
        torch.cuda.synchronize()
        assert torch.equal(a, b), p


def test_fused_rejects_bad_arguments():
    x = _img(8, 8, torch.uint8, seed=1)
    xi = api.image(x)
    p = api.Params().c()
    assert B.weno_zoom2x_cascade_workspace_bytes(xi, 0, p) == 0
    assert B.weno_zoom2x_cascade_workspace_bytes(xi, B.WENO_CASCADE_MAX_LEVELS + 1, p) == 0
    need = B.weno_zoom2x_cascade_workspace_bytes(xi, 2, p)
    assert need > 0
    out = torch.empty(3, 32, 32, dtype=torch.uint8, device=DEV)
    ws = torch.empty(need + 256, dtype=torch.uint8, device=DEV)
    base = (ws.data_ptr() + 255) & ~255
    oi = api.image(out)
    s = api._stream(x.device)
    assert B.weno_zoom2x_cascade(xi, 0, oi, 0, 2, p, base, need, s) == B.WENO_OK
    assert B.weno_zoom2x_cascade(xi, 0, oi, 0, 3, p, base, need, s) == B.WENO_EINVAL  # shape
    assert B.weno_zoom2x_cascade(xi, 0, oi, 0, 2, p, base, need - 1, s) == B.WENO_EWORKSPACE
    assert B.weno_zoom2x_cascade(xi, 0, oi, 0, 2, p, base + 16, need, s) == B.WENO_EWORKSPACE
    assert B.weno_zoom2x_cascade(xi, 0, oi, 0, 2, p, None, need, s) == B.WENO_EWORKSPACE
    torch.cuda.synchronize()
