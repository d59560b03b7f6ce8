"""Batched persistent launch: each image equals the single-image kernel bit
for bit, CUDA-graph replay equals direct launches, malformed descriptors are
skipped, and sampled windows match the oracle."""
import ctypes

import numpy as np
import pytest
import torch

import parity
from paper_2312_00229_gb300 import api, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"

SIZES = [(1, 1), (1, 300), (300, 1), (64, 64), (65, 241), (500, 700), (97, 1024), (1024, 97),
         (3, 5), (256, 480)]


def _images(dtype=torch.uint8, sizes=SIZES, seed=0):
    g = torch.Generator(device=DEV).manual_seed(seed)
    imgs = []
    for (h, w) in sizes:
        t = torch.randint(0, 256, (3, h, w), device=DEV, generator=g, dtype=torch.uint8)
        if dtype == torch.uint8:
            imgs.append(t)
        else:
            imgs.append((t.float() / 255.0).to(dtype))
    return imgs


@pytest.mark.parametrize("dtype", [torch.uint8, torch.float16, torch.float32])
@pytest.mark.parametrize("rows", [0, 16])
def test_batched_equals_single(dtype, rows):
    imgs = _images(dtype)
    outs = api.zoom2x_batched(imgs, rows_per_tile=rows)
    singles = [api.zoom2x_fwd(x, rows_per_tile=rows) for x in imgs]
    torch.cuda.synchronize()
    for o, s in zip(outs, singles):
        assert torch.equal(o, s)


def test_batched_out_mode_and_layout():
    imgs = [x.permute(1, 2, 0).contiguous() for x in _images(torch.uint8, SIZES[:6], seed=3)]
    prm = api.Params(out_mode=1)
    outs = api.zoom2x_batched(imgs, prm, layout="hwc")
    singles = [api.zoom2x_fwd(x, prm, layout="hwc") for x in imgs]
    torch.cuda.synchronize()
    for o, s in zip(outs, singles):
        assert torch.equal(o, s)


def test_batched_graph_replay():
    imgs = _images(torch.float16, seed=5)
    plan = api.BatchedPlan(imgs, out_dtype=torch.float16)
    plan.run()  # warm-up outside capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    for seed in (11, 12):
        new = _images(torch.float16, seed=seed)
        for dst, src in zip(plan.inputs, new):
            dst.copy_(src)
        for o in plan.outputs:
            o.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for x, o in zip(plan.inputs, plan.outputs):
            assert torch.equal(o, api.zoom2x_fwd(x))


def test_batched_skips_malformed_descriptor():
    imgs = _images(torch.uint8, SIZES[:4], seed=8)
    outs = [api._out_like(x, api.Params(), "chw", torch.uint8).fill_(77) for x in imgs]
    bad = torch.full((3, 9, 9), 77, dtype=torch.uint8, device=DEV)  # wrong shape for image 1
    outs[1] = bad
    plan = api.BatchedPlan(imgs, outputs=outs)
    plan.run()
    torch.cuda.synchronize()
    assert bool((bad == 77).all())
    for i in (0, 2, 3):
        assert torch.equal(outs[i], api.zoom2x_fwd(imgs[i]))


def test_batched_uneven_scenes_against_oracle():
    """A subset of the 256-image uneven workload (FP16 storage): all images
    checked bit-exact against single launches, a few against the oracle."""
    sizes = scenes.uneven_sizes()[:24]
    imgs = scenes.uneven_batch(24)
    xs = [torch.from_numpy(scenes.planar(im)).to(DEV).float().div(255).half() for im in imgs]
    outs = api.zoom2x_batched(xs)
    torch.cuda.synchronize()
    for x, o in zip(xs, outs):
        assert torch.equal(o, api.zoom2x_fwd(x))
    for k in (0, 1, 5):
        h, w = sizes[k]
        A = parity.decode(xs[k][:, : min(h, 40), : min(w, 50)].cpu())
        ref = parity.oracle_planes(A, api.Params())
        hh, ww = min(h, 40) - 6, min(w, 50) - 6
        if hh > 0 and ww > 0:
            parity.compare(outs[k][:, : 2 * hh, : 2 * ww].cpu(), ref[:, : 2 * hh, : 2 * ww],
                           "f16")


@pytest.mark.parametrize("dtype", [torch.uint8, torch.bfloat16])
def test_batched_mixed_layouts(dtype):
    """One call whose images mix layouts: unit column stride (including rows
    at odd byte offsets) and column stride 2; each equals the single-image
    kernel bit for bit."""
    base = _images(dtype, [(37, 251), (64, 97), (5, 513), (130, 256), (1, 3)], seed=11)
    imgs = []
    for i, x in enumerate(base):
        if i % 2:
            wide = torch.zeros(x.shape[:-1] + (2 * x.shape[-1],), device=DEV, dtype=dtype)
            wide[..., ::2] = x
            imgs.append(wide[..., ::2])
        else:
            imgs.append(x[:, :, 1:] if x.shape[-1] > 1 else x)  # rows start off 16-byte blocks
    outs = api.zoom2x_batched(imgs)
    singles = [api.zoom2x_fwd(x) for x in imgs]
    torch.cuda.synchronize()
    for o, s in zip(outs, singles):
        assert torch.equal(o, s)


def test_batched_fp32_with_data_bound():
    """FP32 images with a caller's bound take the direct-weight batched
    kernel; each equals the single-image kernel with the same parameters bit
    for bit, and stays within FP32 rounding of the unbounded (scale-free)
    result."""
    imgs = _images(torch.float32, SIZES[:7], seed=13)
    prm = api.Params(data_bound=1.0)
    outs = api.zoom2x_batched(imgs, prm)
    singles = [api.zoom2x_fwd(x, prm) for x in imgs]
    plain = [api.zoom2x_fwd(x) for x in imgs]
    torch.cuda.synchronize()
    for o, s, q in zip(outs, singles, plain):
        assert torch.equal(o, s)
        assert (o - q).abs().max().item() <= 4e-6


@pytest.mark.parametrize("dtype", [torch.uint8, torch.float16, torch.float32])
@pytest.mark.parametrize("tw", [119, 246, 118])
def test_batched_other_tile_shapes(dtype, tw):
    """The persistent launch with 128-thread CTAs (tile width 119) or two
    columns per thread (246: 128 threads, 118: 64) equals the single-image
    kernel bit for bit for every image, edge sizes included."""
    imgs = _images(dtype, SIZES, seed=17)
    for rows in (0, 32):
        outs = api.BatchedPlan(imgs, rows_per_tile=rows, tile_width=tw).run()
        singles = [api.zoom2x_fwd(x) for x in imgs]
        torch.cuda.synchronize()
        for x, o, s in zip(imgs, outs, singles):
            assert torch.equal(o, s), (tuple(x.shape), rows, tw)
    from paper_2312_00229_gb300 import binding as B
    plan = api.BatchedPlan(imgs[:2])
    for tw in (1, 117, 120, 256):
        rc = B.weno_zoom2x_batched(2, ctypes.c_void_p(plan.d_in.data_ptr()), plan.in_t,
                                   ctypes.c_void_p(plan.d_out.data_ptr()), plan.out_t,
                                   plan.params.c(), ctypes.c_void_p(plan.workspace.data_ptr()),
                                   plan.ws_bytes, 0, tw, api._stream(plan.device))
        assert rc == B.WENO_EINVAL, tw
