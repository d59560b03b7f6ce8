"""PyTorch-facing API of the WD WENO 2x zoom (arXiv 2312.00229, Sec. 3).

PyTorch supplies device memory and streams; every step of the method runs in
``libwdweno.so``.  Tensors must live on a CUDA device; there is no CPU path.

Layouts: ``"chw"`` = [C, H, W] (also [N, C, H, W] and [H, W]), ``"hwc"`` =
[H, W, C] (interleaved pixels).  Any strides are accepted.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional, Sequence

import torch

from . import binding as B

_DT = {torch.uint8: B.WENO_U8, torch.float16: B.WENO_F16, torch.bfloat16: B.WENO_BF16,
       torch.float32: B.WENO_F32}


@dataclasses.dataclass(frozen=True)
class Params:
    """Parameters of the method (``weno_params``).

    beta  : exponent of Eq. (alpha) (Sec. 4 uses 2)
    k_eps : eps_h = k_eps h^2 (Sec. 2: 1e-8)
    h     : coarse grid spacing (1 = pixel units)
    si_scale : 0 normalized indicator length scale, 1 literal sqrt(2) h
    out_mode : 0 -> 2n x 2m output, 1 -> (2n-1) x (2m-1) (Sec. 3)
    clamp_float : saturate float outputs to [0, 1]
    data_bound : 0, or a bound on |input| the caller guarantees (lets the
                 library take the direct beta = 2 weights for FP32/BF16 data)
    nbr_c : neighbour weight nbr_c h^2 of D in both phases (h^2/8: the
            reading of Eqs. 2DsmoothnessFinal/tezine that reproduces Table 1)
    """
    beta: float = 2.0
    k_eps: float = 1e-8
    h: float = 1.0
    si_scale: int = B.WENO_SI_NORMALIZED
    out_mode: int = B.WENO_OUT_2N
    clamp_float: bool = False
    data_bound: float = 0.0
    nbr_c: float = 0.125

    def c(self) -> B.weno_params:
        p = B.weno_params()
        p.beta, p.k_eps, p.h = float(self.beta), float(self.k_eps), float(self.h)
        p.si_scale, p.out_mode, p.clamp_float = int(self.si_scale), int(self.out_mode), int(
            bool(self.clamp_float))
        p.data_bound = float(self.data_bound)
        p.nbr_c = float(self.nbr_c)
        return p


def lib():
    return B.load()


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _require_cuda(t: torch.Tensor, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if t.dtype not in _DT:
        raise TypeError(f"{name}: unsupported dtype {t.dtype}")


def _planes(t: torch.Tensor, layout: str):
    """(height, width, channels, stride_c, stride_h, stride_w) of a tensor,
    folding a leading batch dimension into the channel count when the planes
    are uniformly strided."""
    if t.dim() == 2:
        return t.shape[0], t.shape[1], 1, 1, t.stride(0), t.stride(1)
    if layout == "hwc":
        if t.dim() != 3:
            raise ValueError("hwc layout needs a 3-D tensor [H, W, C]")
        return t.shape[0], t.shape[1], t.shape[2], t.stride(2), t.stride(0), t.stride(1)
    if t.dim() == 3:
        return t.shape[1], t.shape[2], t.shape[0], t.stride(0), t.stride(1), t.stride(2)
    if t.dim() == 4:
        N, C = t.shape[0], t.shape[1]
        if N == 1 or C == 1 or t.stride(0) == C * t.stride(1):
            sc = t.stride(1) if C > 1 else t.stride(0)
            return t.shape[2], t.shape[3], N * C, max(sc, 1), t.stride(2), t.stride(3)
        raise ValueError("4-D input needs uniformly strided planes (e.g. contiguous NCHW)")
    raise ValueError("expected a 2-D, 3-D or 4-D tensor")


def image(t: torch.Tensor, layout: str = "chw") -> B.weno_image:
    h, w, c, sc, sh, sw = _planes(t, layout)
    im = B.weno_image()
    im.data = t.data_ptr()
    im.height, im.width, im.channels = int(h), int(w), int(c)
    im.stride_c, im.stride_h, im.stride_w = int(max(sc, 1)), int(max(sh, 1)), int(max(sw, 1))
    return im


def out_hw(h: int, w: int, params: Params):
    d = 1 if params.out_mode == B.WENO_OUT_2N_MINUS_1 else 0
    return 2 * h - d, 2 * w - d


def _out_like(x: torch.Tensor, params: Params, layout: str, dtype) -> torch.Tensor:
    shape = list(x.shape)
    if layout == "hwc":
        shape[0], shape[1] = out_hw(shape[0], shape[1], params)
    else:
        shape[-2], shape[-1] = out_hw(shape[-2], shape[-1], params)
    return torch.empty(shape, dtype=dtype, device=x.device)


def zoom2x_fwd(x: torch.Tensor, params: Optional[Params] = None, out_dtype=None,
               layout: str = "chw", rows_per_tile: Optional[int] = None,
               out: Optional[torch.Tensor] = None, tile_width: int = 0) -> torch.Tensor:
    """Forward 2x zoom (``weno_zoom2x_fwd``); no autograd.

    ``rows_per_tile``: band height per CTA; None = the autotuner's cached
    choice for this size class (see ``autotune``), 0 = the library default.
    ``tile_width``: output columns per CTA, 247 (256 threads) or 119 (128
    threads); 0 = the library's choice for the image width."""
    params = params or Params()
    _require_cuda(x, "x")
    if x.numel() == 0:
        raise ValueError("empty input")
    if out is None:
        out = _out_like(x, params, layout, out_dtype or x.dtype)
    _require_cuda(out, "out")
    if rows_per_tile is None:
        from . import autotune
        rows_per_tile = autotune.lookup(x, out.dtype, layout)
        if tile_width == 0:
            tile_width = autotune.lookup_width(x, out.dtype, layout)
    rc = B.weno_zoom2x_fwd_tiled(image(x, layout), _DT[x.dtype], image(out, layout),
                                 _DT[out.dtype], params.c(), rows_per_tile, int(tile_width),
                                 _stream(x.device))
    B.check("weno_zoom2x_fwd", rc)
    return out


def zoom2x_bwd(x: torch.Tensor, grad_out: torch.Tensor, params: Optional[Params] = None,
               layout: str = "chw", workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Input gradient of the zoom for FP32 data (``weno_zoom2x_bwd``)."""
    params = params or Params()
    _require_cuda(x, "x")
    _require_cuda(grad_out, "grad_out")
    if x.dtype != torch.float32 or grad_out.dtype != torch.float32:
        raise TypeError("the adjoint runs on FP32 data")
    grad_in = torch.empty_like(x)
    xi = image(x, layout)
    need = B.weno_zoom2x_bwd_workspace_bytes(xi)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=x.device)
    rc = B.weno_zoom2x_bwd(xi, image(grad_out, layout), image(grad_in, layout), params.c(),
                           ctypes.c_void_p(workspace.data_ptr()), need, _stream(x.device))
    B.check("weno_zoom2x_bwd", rc)
    return grad_in


class WenoZoom2x(torch.autograd.Function):
    """Differentiable WD WENO 2x zoom; backward is the hand-written adjoint."""

    @staticmethod
    def forward(ctx, x, params, layout):
        ctx.params, ctx.layout = params, layout
        ctx.save_for_backward(x)
        return zoom2x_fwd(x, params, layout=layout)

    @staticmethod
    def backward(ctx, grad_out):
        (x,) = ctx.saved_tensors
        g = zoom2x_bwd(x, grad_out.contiguous(), ctx.params, ctx.layout)
        return g, None, None


def zoom2x(x: torch.Tensor, params: Optional[Params] = None, out_dtype=None,
           layout: str = "chw") -> torch.Tensor:
    """2x zoom; differentiable for FP32 inputs that require grad."""
    params = params or Params()
    if torch.is_grad_enabled() and x.requires_grad:
        if x.dtype != torch.float32 or (out_dtype not in (None, torch.float32)):
            raise TypeError("gradients are supported for FP32 in and out")
        return WenoZoom2x.apply(x, params, layout)
    return zoom2x_fwd(x, params, out_dtype=out_dtype, layout=layout)


_TYPE_BOUND = {torch.uint8: 1.0, torch.float16: 65504.0}
# One 2x level maps data bounded by M to data bounded by 1.5625 M: an x value
# is a convex combination of quadratic interpolants (|p| <= 1.25 max|node|),
# and a "+" value one of interpolants whose nodes include x values.  The
# factor carries slack for the rounding of the weights.
_LEVEL_GROWTH = 1.5625 * (1.0 + 1e-3)


def _level_bounds(x: torch.Tensor, params: Params, levels: int):
    """Bound on |input| of each level of a chain of 2x zooms (and of the
    level after the last), from the input's storage type and the caller's
    ``data_bound``; 0 where neither bounds the data."""
    b0 = _TYPE_BOUND.get(x.dtype, 0.0)
    if params.data_bound > 0 and (b0 == 0.0 or params.data_bound < b0):
        b0 = float(params.data_bound)
    return [b0 * _LEVEL_GROWTH ** lvl for lvl in range(levels + 1)]


def cascade_zoom(x: torch.Tensor, levels: int, params: Optional[Params] = None, out_dtype=None,
                 inter_dtype=torch.float32, layout: str = "chw",
                 fused: bool = False) -> torch.Tensor:
    """``levels`` successive 2x zooms (Sec. 3.3, Eq. zoomfactor); the
    intermediate images are kept in ``inter_dtype`` and only the last one is
    encoded to ``out_dtype``.  Each level's coarse grid is the previous
    level's fine grid, so its spacing ``h`` is half the previous one.  The
    bound the input's type gives is carried to the later levels
    (``data_bound``), so FP32 intermediates keep the direct weights.

    ``fused=True`` runs every level in one persistent launch
    (``weno_zoom2x_cascade``; FP32 intermediates in a workspace) with the
    same result."""
    params = params or Params()
    if fused:
        if inter_dtype != torch.float32:
            raise ValueError("the fused cascade keeps FP32 intermediates")
        _require_cuda(x, "x")
        n, m = _hw(x, layout)
        d = 1 if params.out_mode == B.WENO_OUT_2N_MINUS_1 else 0
        oh, ow = n, m
        for _ in range(levels):
            oh, ow = 2 * oh - d, 2 * ow - d
        shape = list(x.shape)
        if layout == "hwc":
            shape[0], shape[1] = oh, ow
        else:
            shape[-2], shape[-1] = oh, ow
        out = torch.empty(shape, dtype=out_dtype or x.dtype, device=x.device)
        xi, oi, pc = image(x, layout), image(out, layout), params.c()
        nbytes = B.weno_zoom2x_cascade_workspace_bytes(xi, levels, pc)
        if nbytes == 0:
            raise ValueError("malformed cascade request")
        ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=x.device)
        base = (ws.data_ptr() + 255) & ~255
        B.check("weno_zoom2x_cascade",
                B.weno_zoom2x_cascade(xi, _DT[x.dtype], oi, _DT[out.dtype], levels, pc, base,
                                      nbytes, _stream(x.device)))
        return out
    bounds = _level_bounds(x, params, levels)
    cur = x
    for lvl in range(levels):
        last = lvl == levels - 1
        p = dataclasses.replace(params, h=params.h / (1 << lvl), data_bound=bounds[lvl])
        cur = zoom2x_fwd(cur, p, out_dtype=(out_dtype or x.dtype) if last else inter_dtype,
                         layout=layout)
    return cur


def _hw(t: torch.Tensor, layout: str):
    h, w, _, _, _, _ = _planes(t, layout)
    return int(h), int(w)


def resample(x: torch.Tensor, out_h: int, out_w: int, params: Optional[Params] = None,
             out_dtype=None, layout: str = "chw", out: Optional[torch.Tensor] = None):
    """Tensor-product WENO resampling (Sec. 3.3, Eq. tensor) to any
    ``out_h x out_w`` on endpoint-aligned grids (``weno_resample``).
    ``params.h`` is the spacing of the input grid; ``out_mode`` and
    ``si_scale`` do not apply."""
    params = params or Params()
    _require_cuda(x, "x")
    if x.numel() == 0 or out_h < 1 or out_w < 1:
        raise ValueError("empty input or output")
    if out is None:
        shape = list(x.shape)
        if layout == "hwc":
            shape[0], shape[1] = out_h, out_w
        else:
            shape[-2], shape[-1] = out_h, out_w
        out = torch.empty(shape, dtype=out_dtype or x.dtype, device=x.device)
    _require_cuda(out, "out")
    rc = B.weno_resample(image(x, layout), _DT[x.dtype], image(out, layout), _DT[out.dtype],
                         params.c(), _stream(x.device))
    B.check("weno_resample", rc)
    return out


def zoom_levels(n: int, m: int, out_h: int, out_w: int) -> int:
    """Doublings on the (2n-1) grid (Eq. zoomfactor: n -> 2^k (n-1) + 1)
    until both sides reach the target (sides of one sample never grow)."""
    k = 0
    while (n > 1 and n < out_h) or (m > 1 and m < out_w):
        n, m, k = 2 * n - 1, 2 * m - 1, k + 1
    return k


def zoom_to(x: torch.Tensor, out_h: int, out_w: int, params: Optional[Params] = None,
            out_dtype=None, inter_dtype=torch.float32, layout: str = "chw") -> torch.Tensor:
    """Arbitrary-resolution zoom (Sec. 3.3): k WD WENO doublings on the
    (2n-1) grid up to the first size that covers the target, then tensor
    WENO resampling down to ``out_h x out_w`` (the 3x example zooms n to
    4n-3, then resamples to 3n)."""
    params = params or Params()
    n, m = _hw(x, layout)
    k = zoom_levels(n, m, out_h, out_w)
    bounds = _level_bounds(x, params, k)
    cur = x
    p = dataclasses.replace(params, out_mode=B.WENO_OUT_2N_MINUS_1)
    for lvl in range(k):
        cur = zoom2x_fwd(cur, dataclasses.replace(p, h=params.h / (1 << lvl),
                                                  data_bound=bounds[lvl]),
                         out_dtype=inter_dtype, layout=layout)
    return resample(cur, out_h, out_w,
                    dataclasses.replace(params, h=params.h / (1 << k), data_bound=bounds[k]),
                    out_dtype=out_dtype or x.dtype, layout=layout)


class BatchedPlan:
    """Device-resident descriptors, outputs and workspace of one batched call
    (``weno_zoom2x_batched``).  ``run()`` enqueues the single persistent
    launch; it can be captured into a CUDA graph and replayed."""

    def __init__(self, images: Sequence[torch.Tensor], params: Optional[Params] = None,
                 out_dtype=None, layout: str = "chw", rows_per_tile: int = 0,
                 outputs: Optional[Sequence[torch.Tensor]] = None, tile_width: int = 0):
        if len(images) == 0:
            raise ValueError("empty batch")
        self.params = params or Params()
        self.layout = layout
        self.rows_per_tile = int(rows_per_tile)
        self.tile_width = int(tile_width)  # 0 = 247, or 119 (128-thread CTAs)
        dev = images[0].device
        in_dt = images[0].dtype
        for im in images:
            _require_cuda(im, "image")
            if im.dtype != in_dt or im.device != dev:
                raise ValueError("all images must share dtype and device")
        self.inputs = list(images)
        odt = out_dtype or in_dt
        self.outputs = list(outputs) if outputs is not None else [
            _out_like(im, self.params, layout, odt) for im in images]
        self.in_t, self.out_t = _DT[in_dt], _DT[self.outputs[0].dtype]
        n = len(images)
        host_in = (B.weno_image * n)(*[image(t, layout) for t in self.inputs])
        host_out = (B.weno_image * n)(*[image(t, layout) for t in self.outputs])
        nbytes = ctypes.sizeof(B.weno_image) * n
        self.d_in = torch.frombuffer(bytearray(bytes(host_in)), dtype=torch.uint8).to(dev)
        self.d_out = torch.frombuffer(bytearray(bytes(host_out)), dtype=torch.uint8).to(dev)
        assert self.d_in.numel() == nbytes
        self.ws_bytes = B.weno_zoom2x_batched_workspace_bytes(n)
        self.workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.count = n
        self.device = dev

    def run(self) -> List[torch.Tensor]:
        rc = B.weno_zoom2x_batched(self.count, ctypes.c_void_p(self.d_in.data_ptr()), self.in_t,
                                   ctypes.c_void_p(self.d_out.data_ptr()), self.out_t,
                                   self.params.c(), ctypes.c_void_p(self.workspace.data_ptr()),
                                   self.ws_bytes, self.rows_per_tile, self.tile_width,
                                   _stream(self.device))
        B.check("weno_zoom2x_batched", rc)
        return self.outputs


def zoom2x_batched(images: Sequence[torch.Tensor], params: Optional[Params] = None,
                   out_dtype=None, layout: str = "chw", rows_per_tile: Optional[int] = None):
    """Zooms images of independent sizes in one persistent launch."""
    tile_width = 0
    if rows_per_tile is None:
        from . import autotune
        rows_per_tile, tile_width = autotune.lookup_batched(images, out_dtype, layout)
    return BatchedPlan(images, params, out_dtype, layout, rows_per_tile,
                       tile_width=tile_width).run()


class HostPipeline:
    """Zooms a stream of frames that live in (pinned) host memory, overlapping
    the copy of frame i+1 to the GPU, the zoom of frame i and the copy of
    frame i-1 back to the host on three CUDA streams, with `depth` device
    buffer pairs in flight.

        pipe = HostPipeline((3, 1080, 1920), torch.uint8, device="cuda")
        for x_host, y_host in frames:          # pinned CPU tensors
            pipe.submit(x_host, y_host)
        pipe.flush()                           # all y_host written

    `x_host` must stay unchanged and `y_host` unread until flush() (or until
    `depth` later submissions have been made, when that frame's buffers are
    reused).  Shapes and dtypes are fixed per pipeline."""

    def __init__(self, in_shape, in_dtype, params: Optional[Params] = None, out_dtype=None,
                 layout: str = "chw", device="cuda", depth: int = 3):
        self.params = params or Params()
        self.layout = layout
        self.device = torch.device(device)
        self.depth = int(depth)
        self.xd = [torch.empty(in_shape, dtype=in_dtype, device=self.device)
                   for _ in range(self.depth)]
        self.od = [_out_like(x, self.params, layout, out_dtype or in_dtype) for x in self.xd]
        self.s_in = torch.cuda.Stream(self.device)
        self.s_run = torch.cuda.Stream(self.device)
        self.s_out = torch.cuda.Stream(self.device)
        ev = lambda: [torch.cuda.Event() for _ in range(self.depth)]
        self.e_in, self.e_run, self.e_out = ev(), ev(), ev()
        self.used = [False] * self.depth
        self.i = 0

    @property
    def out_shape(self):
        return tuple(self.od[0].shape)

    def submit(self, x_host: torch.Tensor, y_host: torch.Tensor) -> None:
        k = self.i % self.depth
        xd, od = self.xd[k], self.od[k]
        with torch.cuda.stream(self.s_in):
            if self.used[k]:
                self.s_in.wait_event(self.e_run[k])   # xd[k] read by the previous zoom
            xd.copy_(x_host, non_blocking=True)
            self.e_in[k].record(self.s_in)
        with torch.cuda.stream(self.s_run):
            self.s_run.wait_event(self.e_in[k])
            if self.used[k]:
                self.s_run.wait_event(self.e_out[k])  # od[k] copied out
            zoom2x_fwd(xd, self.params, layout=self.layout, out=od)
            self.e_run[k].record(self.s_run)
        with torch.cuda.stream(self.s_out):
            self.s_out.wait_event(self.e_run[k])
            y_host.copy_(od, non_blocking=True)
            self.e_out[k].record(self.s_out)
        self.used[k] = True
        self.i += 1

    def flush(self) -> None:
        self.s_out.synchronize()
