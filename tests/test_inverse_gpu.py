"""Inverse problem through the differentiable zoom: recover a 256x256 RGB
image from its 512x512 WD WENO zoom with 200 Adam steps (lr 1e-2, start at
zero).  The same optimisation run through the FP64 autograd restatement of
the oracle gives the reference PSNRs."""
import numpy as np
import pytest
import torch

from oracle import wdweno_torch
from paper_2312_00229_gb300 import api, scenes

pytestmark = pytest.mark.gpu

STEPS, LR = 200, 1e-2


def _psnr(a, b):
    return float(10.0 * np.log10(1.0 / float(((a - b) ** 2).mean())))


def _recover(zoom, x_true, T):
    x = torch.zeros_like(x_true, requires_grad=True)
    opt = torch.optim.Adam([x], lr=LR)
    for _ in range(STEPS):
        opt.zero_grad()
        loss = ((zoom(x) - T) ** 2).sum()
        loss.backward()
        opt.step()
    with torch.no_grad():
        return _psnr(x, x_true), _psnr(zoom(x), T)


def test_adam_recovers_low_res_image():
    img = scenes.piecewise_smooth(256, 256, seed=scenes.seed_for(5, 1))
    x64 = torch.from_numpy(scenes.planar(img).astype(np.float64) / 255.0)
    with torch.no_grad():
        T64 = wdweno_torch.zoom2x(x64)
    ref_x, ref_z = _recover(wdweno_torch.zoom2x, x64, T64)

    x32 = x64.float().cuda()
    T32 = T64.float().cuda()
    got_x, got_z = _recover(lambda v: api.zoom2x(v), x32, T32)
    # the FP64 run reaches about 36 dB (image) and 40 dB (zoom)
    assert ref_x > 30.0 and ref_z > 34.0
    assert abs(got_x - ref_x) < 1.0, (got_x, ref_x)
    assert abs(got_z - ref_z) < 1.0, (got_z, ref_z)
