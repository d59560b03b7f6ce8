"""Tensor-WENO resampling and the arbitrary-scale zoom (Sec. 3.3): CUDA path
through the C ABI against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2312_00229_gb300 import api, scenes

pytestmark = pytest.mark.gpu

DEV = "cuda"
RNG = np.random.default_rng(20231203)


def _resample(A01, oh, ow, in_dt="f32", out_dt="f32", params=api.Params(), layout="chw"):
    x = parity.encode(A01, in_dt)
    if layout == "hwc":
        x = x.permute(1, 2, 0).contiguous()
    out = api.resample(x.to(DEV), oh, ow, params, out_dtype=parity.TORCH_DT[out_dt],
                       layout=layout)
    torch.cuda.synchronize()
    if layout == "hwc":
        out, x = out.permute(2, 0, 1), x.permute(2, 0, 1)
    ref = oracle.tensor_resample(parity.decode(x), oh, ow, beta=params.beta,
                                 k_eps=params.k_eps, h=params.h)
    return out, ref


SIZES = [((1, 1), (1, 1)), ((1, 1), (5, 3)), ((1, 17), (1, 40)), ((23, 1), (7, 1)),
         ((2, 3), (9, 11)), ((7, 9), (7, 9)), ((64, 64), (192, 192)), ((65, 241), (97, 700)),
         ((130, 481), (45, 160)), ((33, 500), (100, 1499)), ((300, 7), (1000, 2))]


@pytest.mark.parametrize("src,dst", SIZES)
def test_resample_f32_sizes(src, dst):
    A = RNG.random((2,) + src)
    out, ref = _resample(A, *dst)
    parity.compare(out, ref, "f32")


@pytest.mark.parametrize("beta", [0.0, 0.1, 1.0, 2.0, 3.0])
def test_resample_beta(beta):
    img = scenes.piecewise_smooth(61, 83, seed=scenes.seed_for(6, 1), scale_features=True)
    A = scenes.planar(img).astype(np.float64) / 255.0
    out, ref = _resample(A, 150, 211, params=api.Params(beta=beta))
    parity.compare(out, ref, "f32")


@pytest.mark.parametrize("in_dt,out_dt", [("u8", "u8"), ("f16", "f16"), ("bf16", "bf16"),
                                          ("u8", "f32"), ("f32", "u8")])
def test_resample_storage_types(in_dt, out_dt):
    img = scenes.pixel_art(48, 40, seed=scenes.seed_for(6, 2))
    A = scenes.planar(img).astype(np.float64) / 255.0
    out, ref = _resample(A, 144, 120, in_dt, out_dt)
    parity.compare(out, ref, out_dt)


def test_resample_hwc_and_params():
    A = RNG.random((3, 50, 70))
    p = api.Params(k_eps=0.5, h=0.25)
    out, ref = _resample(A, 77, 31, params=p, layout="hwc")
    parity.compare(out, ref, "f32")


def test_resample_strided_view_and_range():
    """A cropped view in, a non-unit-range FP32 image."""
    big = torch.from_numpy(RNG.normal(size=(2, 80, 90)).astype(np.float32) * 40.0)
    view = big[:, 5:70, 3:81]
    out = api.resample(view.to(DEV)[:, :, :], 100, 123)
    torch.cuda.synchronize()
    ref = oracle.tensor_resample(view.double().numpy(), 100, 123)
    rng = float(ref.max() - ref.min())
    parity.compare(out, ref, "f32", value_range=rng)


@pytest.mark.parametrize("shape,target", [((24, 20), (72, 60)), ((17, 33), (50, 98)),
                                          ((40, 40), (57, 61)), ((9, 13), (200, 150))])
def test_zoom_to_matches_oracle(shape, target):
    A = RNG.random((2,) + shape)
    x = torch.from_numpy(A.astype(np.float32)).to(DEV)
    out = api.zoom_to(x, *target)
    torch.cuda.synchronize()
    ref = oracle.zoom_to(A.astype(np.float32).astype(np.float64), *target)
    # FP32 rounding of each intermediate level adds up: one FP32 tolerance
    # per level plus the resampling
    k = api.zoom_levels(shape[0], shape[1], *target)
    g = out.cpu().double().numpy()
    assert g.shape == ref.shape
    assert np.abs(g - ref).max() <= parity.F32_TOL * (k + 1)


def test_zoom_to_3x_pixel_art_u8():
    """The 3x example of Sec. 3.3 on a pixel-art image, uint8 in and out."""
    img = scenes.pixel_art(64, 48, seed=scenes.seed_for(6, 3))
    x = torch.from_numpy(np.ascontiguousarray(scenes.planar(img))).to(DEV)
    out = api.zoom_to(x, 192, 144)
    torch.cuda.synchronize()
    ref = oracle.zoom_to(scenes.planar(img).astype(np.float64) / 255.0, 192, 144)
    want = oracle.encode_u8(ref).astype(np.int64)
    diff = out.cpu().numpy().astype(np.int64) - want
    assert np.abs(diff).max() <= 1
    scaled = np.clip(ref, 0, 1) * 255.0
    near = np.abs(scaled - np.floor(scaled) - 0.5) <= 3 * parity.TIE_WINDOW
    assert np.all(near[diff != 0])


def test_resample_full_size_sampled():
    """4K RGB u8 -> 3x (11520 x 6480): sampled outputs against the oracle's
    1-D interpolants evaluated one by one."""
    img = scenes.piecewise_smooth(2160, 3840, seed=scenes.seed_for(4, 0))
    x = torch.from_numpy(np.ascontiguousarray(scenes.planar(img))).to(DEV)
    oh, ow = 6480, 11520
    out = api.resample(x, oh, ow, out_dtype=torch.float32)
    torch.cuda.synchronize()
    A = scenes.planar(img).astype(np.float64) / 255.0
    rs = np.concatenate([[0, 1, oh - 1], RNG.integers(0, oh, 60)])
    cs = np.concatenate([[0, ow - 2, ow - 1], RNG.integers(0, ow, 60)])
    g = out[:, torch.from_numpy(rs).to(DEV)][:, :, torch.from_numpy(cs).to(DEV)].cpu().numpy()
    for ri, r in enumerate(rs):
        y = r * 2159 / (oh - 1)
        i0 = min(int(np.floor(y)), 2158)
        lo, hi = max(i0 - 1, 0), min(i0 + 3, 2160)
        for ci, c in enumerate(cs):
            xx = c * 3839 / (ow - 1)
            k0 = min(int(np.floor(xx)), 3838)
            cl, ch = max(k0 - 1, 0), min(k0 + 3, 3840)
            for ch_ in range(3):
                Z = np.zeros(3840)
                for k in range(cl, ch):
                    Z[k] = oracle.weno_spline(A[ch_, lo:hi, k], y - lo)
                want = oracle.weno_spline(Z[cl:ch], xx - cl)
                assert abs(g[ch_, ri, ci] - want) <= parity.F32_TOL, (r, c, ch_)


def test_resample_rejects_bad_arguments():
    x = torch.zeros(1, 8, 8, device=DEV)
    with pytest.raises(ValueError):
        api.resample(x, 0, 5)
    with pytest.raises(Exception):
        api.resample(x, 5, 5, out=torch.zeros(2, 5, 5, device=DEV))  # channel mismatch


def test_resample_weight_forms_at_the_range_limits():
    """beta = 2 weights as C_0 eR^2 : C_1 eL^2 directly for uint8 and FP16
    data (range-bounded), else scaled by the larger indicator: parity on both
    sides, with FP16 data at the ends of its range and vanishing eps."""
    big = scenes.planar(scenes.piecewise_smooth(41, 57, seed=scenes.seed_for(6, 4),
                                                scale_features=True)).astype(np.float64)
    big = (big / 255.0 * 2.0 - 1.0) * 65504.0
    big[0, 5, 3:9] = 65504.0
    big[2, 9, 20:23] = -65504.0
    x = torch.from_numpy(big.astype(np.float16))
    out = api.resample(x.to(DEV), 100, 131, out_dtype=torch.float32)
    torch.cuda.synchronize()
    ref = oracle.tensor_resample(x.double().numpy(), 100, 131)
    parity.compare(out, ref, "f32", value_range=float(ref.max() - ref.min()))
    img = scenes.pixel_art(30, 44, seed=scenes.seed_for(6, 5))
    A = scenes.planar(img).astype(np.float64) / 255.0
    for prm in (api.Params(k_eps=1e-30), api.Params(h=1e-6), api.Params(h=1e-6, k_eps=1e6)):
        for in_dt in ("u8", "f16"):
            out, ref = _resample(A, 90, 131, in_dt, "f32", params=prm)
            parity.compare(out, ref, "f32")


def test_resample_direct_and_scaled_weights_agree():
    """FP16 storage (direct weights) and FP32 storage of the same values
    (scaled weights) agree to a few FP32 rounding steps."""
    x = torch.rand(3, 70, 90, device=DEV).to(torch.float16)
    a = api.resample(x, 209, 270, out_dtype=torch.float32)
    b = api.resample(x.float(), 209, 270, out_dtype=torch.float32)
    torch.cuda.synchronize()
    assert (a - b).abs().max().item() <= 4e-6


def test_resample_positions_past_32_bits():
    """An axis whose position numerators j (m - 1) pass 2^32 (70001 columns
    to 70001: 4.9e9) takes the 64-bit division; the rows take the 32-bit
    multiply-high one.  Both against the oracle."""
    A = RNG.random((1, 2, 70001))
    out, ref = _resample(A, 5, 70001)
    parity.compare(out, ref, "f32")


@pytest.mark.parametrize("dtype", [torch.uint8, torch.float16])
def test_cascade_zoom_matches_oracle(dtype):
    """2^k zoom by successive 2x levels (Sec. 3.3, Eq. zoomfactor), h halving
    per level, FP32 intermediates carrying the input type's bound (direct
    weights): against the oracle applied level by level to the FP32 values
    each level stores; one FP32 tolerance per level."""
    img = scenes.pixel_art(40, 56, seed=scenes.seed_for(6, 7))
    A = scenes.planar(img).astype(np.float64) / 255.0
    x = parity.encode(A, "u8" if dtype == torch.uint8 else "f16").to(DEV)
    out = api.cascade_zoom(x, 3, out_dtype=torch.float32)
    torch.cuda.synchronize()
    cur = parity.decode(x.cpu())
    for lvl in range(3):
        cur = oracle.zoom2x(cur, h=1.0 / (1 << lvl)).astype(np.float32).astype(np.float64)
    g = out.cpu().double().numpy()
    assert g.shape == cur.shape == (3, 320, 448)
    assert np.abs(g - cur).max() <= parity.F32_TOL * 3


def test_resample_fp32_with_data_bound():
    """FP32 input with a caller's bound takes the direct weights: oracle
    parity, and agreement with the scaled weights (no bound) to a few FP32
    rounding steps."""
    A = RNG.random((2, 45, 70))
    out, ref = _resample(A, 130, 201, params=api.Params(data_bound=1.0))
    parity.compare(out, ref, "f32")
    x = torch.from_numpy(A.astype(np.float32)).to(DEV)
    a = api.resample(x, 130, 201, api.Params(data_bound=1.0))
    b = api.resample(x, 130, 201)
    torch.cuda.synchronize()
    assert (a - b).abs().max().item() <= 4e-6


@pytest.mark.parametrize("dt", ["u8", "f16", "f32"])
def test_resample_large_reduction_one_thread_per_output(dt):
    """Reductions below half size per axis take the one-thread-per-output
    form (a 4x4 window read per sample); parity on storage types."""
    img = scenes.piecewise_smooth(400, 600, seed=scenes.seed_for(6, 3), scale_features=True)
    A = scenes.planar(img).astype(np.float64) / 255.0
    for dst in [(90, 130), (100, 290), (190, 140)]:
        out, ref = _resample(A, *dst, dt, dt)
        parity.compare(out, ref, dt)
