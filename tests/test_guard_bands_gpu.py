"""Guard bands around every buffer the library writes (the stand-in for a
memory checker): outputs, grad_in and the workspaces of the adjoint, the
batched launch and the fused cascade are placed inside allocations whose
other bytes hold a poison pattern, and inputs sit at the very end of their
allocation.  After each call the poison must be intact and the written
values must equal those of a call on plain tensors."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2312_00229_gb300 import api
from paper_2312_00229_gb300 import binding as B

pytestmark = pytest.mark.gpu
DEV = "cuda"
GUARD = 4096  # bytes of poison on each side
POISON = 0xA5


def _guarded(nbytes):
    """A uint8 buffer of GUARD + nbytes + GUARD poisoned bytes and the
    address of its middle part (256-byte aligned)."""
    buf = torch.full((GUARD + nbytes + GUARD,), POISON, dtype=torch.uint8, device=DEV)
    return buf


def _intact(buf, nbytes):
    torch.cuda.synchronize()
    head = buf[:GUARD]
    tail = buf[GUARD + nbytes:]
    return bool(torch.all(head == POISON)) and bool(torch.all(tail == POISON))


def _view(buf, shape, dtype):
    """A contiguous tensor of `shape` living in the middle part of `buf`."""
    n = int(np.prod(shape)) * torch.tensor([], dtype=dtype).element_size()
    return buf[GUARD:GUARD + n].view(dtype).view(shape)


def _input_at_end(x):
    """A copy of x placed so that its last byte is the allocation's last."""
    nbytes = x.numel() * x.element_size()
    pad = 64  # keeps the start aligned for every element size
    buf = torch.empty(pad + nbytes, dtype=torch.uint8, device=DEV)
    v = buf[pad:].view(x.dtype).view(x.shape)
    v.copy_(x)
    return v


@pytest.mark.parametrize("dt", [torch.uint8, torch.float16, torch.float32])
@pytest.mark.parametrize("tw", [247, 119, 246, 118])
@pytest.mark.parametrize("mode", [0, 1])
def test_forward_output_guard_bands(dt, tw, mode):
    g = torch.Generator(device=DEV).manual_seed(3)
    x = torch.rand(3, 41, 251, device=DEV, generator=g)
    x = (x * 255).to(torch.uint8) if dt == torch.uint8 else x.to(dt)
    xe = _input_at_end(x)
    p = api.Params(out_mode=mode)
    oh, ow = api.out_hw(41, 251, p)
    nbytes = 3 * oh * ow * x.element_size()
    buf = _guarded(nbytes)
    out = _view(buf, (3, oh, ow), dt)
    api.zoom2x_fwd(xe, p, out=out, tile_width=tw, rows_per_tile=16)
    ref = api.zoom2x_fwd(x, p, tile_width=247)
    assert _intact(buf, nbytes)
    assert torch.equal(out, ref)


def test_adjoint_workspace_and_grad_in_guard_bands():
    g = torch.Generator(device=DEV).manual_seed(4)
    x = _input_at_end(torch.rand(2, 37, 130, device=DEV, generator=g))
    go = _input_at_end(torch.randn(2, 74, 260, device=DEV, generator=g))
    need = B.weno_zoom2x_bwd_workspace_bytes(api.image(x))
    wbuf = _guarded(need)
    ws_ptr = wbuf.data_ptr() + GUARD
    gbytes = 2 * 37 * 130 * 4
    gbuf = _guarded(gbytes)
    gin = _view(gbuf, (2, 37, 130), torch.float32)
    rc = B.weno_zoom2x_bwd(api.image(x), api.image(go), api.image(gin), api.Params().c(),
                           ctypes.c_void_p(ws_ptr), need, api._stream(x.device))
    B.check("weno_zoom2x_bwd", rc)
    assert _intact(wbuf, need) and _intact(gbuf, gbytes)
    assert torch.equal(gin, api.zoom2x_bwd(x, go))


@pytest.mark.parametrize("dt", [torch.uint8, torch.float32])
@pytest.mark.parametrize("dst", [(100, 301), (30, 70), (41, 251)])
def test_resample_output_guard_bands(dt, dst):
    g = torch.Generator(device=DEV).manual_seed(5)
    x = torch.rand(3, 41, 251, device=DEV, generator=g)
    x = (x * 255).to(torch.uint8) if dt == torch.uint8 else x
    xe = _input_at_end(x)
    nbytes = 3 * dst[0] * dst[1] * x.element_size()
    buf = _guarded(nbytes)
    out = _view(buf, (3,) + dst, dt)
    api.resample(xe, dst[0], dst[1], out=out)
    ref = api.resample(x, dst[0], dst[1])
    assert _intact(buf, nbytes)
    assert torch.equal(out, ref)


def test_cascade_output_and_workspace_guard_bands():
    g = torch.Generator(device=DEV).manual_seed(6)
    x = _input_at_end((torch.rand(3, 33, 70, device=DEV, generator=g) * 255).to(torch.uint8))
    levels = 3
    pc = api.Params().c()
    xi = api.image(x)
    need = B.weno_zoom2x_cascade_workspace_bytes(xi, levels, pc)
    wbuf = _guarded(need + 256)
    ws_ptr = (wbuf.data_ptr() + GUARD + 255) & ~255
    lo = ws_ptr - wbuf.data_ptr()
    oh, ow = 33 * 8, 70 * 8
    nbytes = 3 * oh * ow
    obuf = _guarded(nbytes)
    out = _view(obuf, (3, oh, ow), torch.uint8)
    rc = B.weno_zoom2x_cascade(xi, B.WENO_U8, api.image(out), B.WENO_U8, levels, pc,
                               ctypes.c_void_p(ws_ptr), need, api._stream(x.device))
    B.check("weno_zoom2x_cascade", rc)
    torch.cuda.synchronize()
    assert bool(torch.all(wbuf[:lo] == POISON)) and bool(torch.all(wbuf[lo + need:] == POISON))
    assert _intact(obuf, nbytes)
    assert torch.equal(out, api.cascade_zoom(x, levels))


def test_batched_outputs_and_workspace_guard_bands():
    g = torch.Generator(device=DEV).manual_seed(7)
    sizes = [(1, 1), (40, 300), (257, 93), (64, 64), (3, 5)]
    imgs = [_input_at_end(torch.rand(3, h, w, device=DEV, generator=g).half()) for h, w in sizes]
    bufs, outs = [], []
    for h, w in sizes:
        nb = 3 * 2 * h * 2 * w * 2
        b = _guarded(nb)
        bufs.append((b, nb))
        outs.append(_view(b, (3, 2 * h, 2 * w), torch.float16))
    plan = api.BatchedPlan(imgs, outputs=outs, rows_per_tile=32)
    wbuf = _guarded(plan.ws_bytes)
    rc = B.weno_zoom2x_batched(plan.count, ctypes.c_void_p(plan.d_in.data_ptr()), plan.in_t,
                               ctypes.c_void_p(plan.d_out.data_ptr()), plan.out_t,
                               plan.params.c(), ctypes.c_void_p(wbuf.data_ptr() + GUARD),
                               plan.ws_bytes, 32, 0, api._stream(imgs[0].device))
    B.check("weno_zoom2x_batched", rc)
    assert _intact(wbuf, plan.ws_bytes)
    for (b, nb), o, x in zip(bufs, outs, imgs):
        assert _intact(b, nb)
        assert torch.equal(o, api.zoom2x_fwd(x, tile_width=247))
