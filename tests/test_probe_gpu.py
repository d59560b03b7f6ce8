"""The FP32-pipe calibration kernel: its chains give the values a host
recomputation of the same fused multiply-adds gives, and its operation
count matches what it runs."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2312_00229_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_fp32_probe_values():
    blocks, iters = 2, 3
    out = torch.full((blocks * 256,), float("nan"), dtype=torch.float32, device="cuda")
    rc = B.weno_fp32_probe(blocks, iters, ctypes.c_void_p(out.data_ptr()),
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == B.WENO_OK
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(blocks, 256)
    a, b = np.float32(0.999999), np.float32(1e-6)
    t = np.arange(256, dtype=np.float32)
    x = np.stack([t * np.float32(1e-3) + np.float32(j) for j in range(16)])  # [chain, thread]
    for _ in range(iters * 8):
        x = (x.astype(np.float64) * np.float64(a) + np.float64(b)).astype(np.float32)
    want = np.zeros(256, dtype=np.float32)
    for j in range(16):
        want = want + x[j]
    for blk in range(blocks):
        np.testing.assert_allclose(got[blk], want, rtol=1e-6)
