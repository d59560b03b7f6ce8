"""Forward parity: CUDA path (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2312_00229_gb300 import api, scenes

pytestmark = pytest.mark.gpu

DEV = "cuda"
RNG = np.random.default_rng(20231201)


def _run(A01: np.ndarray, in_dt: str, out_dt: str, params=api.Params(), layout="chw",
         rows_per_tile=0):
    """A01: float planes [C, H, W] in [0, 1] (or any range for f32)."""
    x = parity.encode(A01, in_dt)
    if layout == "hwc":
        x = x.permute(1, 2, 0).contiguous()
    xd = x.to(DEV)
    out = api.zoom2x_fwd(xd, params, out_dtype=parity.TORCH_DT[out_dt], layout=layout,
                         rows_per_tile=rows_per_tile)
    torch.cuda.synchronize()
    if layout == "hwc":
        out = out.permute(2, 0, 1)
        x = x.permute(2, 0, 1)
    ref = parity.oracle_planes(parity.decode(x), params)
    return out, ref


SHAPES = [(1, 1), (1, 17), (23, 1), (2, 3), (5, 7), (64, 64), (65, 241), (130, 481),
          (33, 500), (7, 719)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", [0, 1])
def test_fwd_f32_random_sizes(shape, mode):
    A = RNG.random((2,) + shape)
    out, ref = _run(A, "f32", "f32", api.Params(out_mode=mode))
    parity.compare(out, ref, "f32")


DTS = ["u8", "f16", "bf16", "f32"]


@pytest.mark.parametrize("in_dt", DTS)
@pytest.mark.parametrize("out_dt", DTS)
def test_fwd_storage_types(in_dt, out_dt):
    img = scenes.piecewise_smooth(37, 300, seed=scenes.seed_for(4, 7), scale_features=True)
    A = scenes.planar(img).astype(np.float64) / 255.0
    out, ref = _run(A, in_dt, out_dt)
    parity.compare(out, ref, out_dt)


@pytest.mark.parametrize("beta", [0.0, 0.1, 1.0, 1.5, 3.0])
def test_fwd_beta(beta):
    A = RNG.random((1, 40, 250))
    out, ref = _run(A, "f32", "f32", api.Params(beta=beta))
    parity.compare(out, ref, "f32")


def test_fwd_literal_si_scale_and_h():
    A = RNG.random((1, 29, 243))
    for prm in (api.Params(si_scale=1), api.Params(h=1 / 64), api.Params(h=0.37, si_scale=1),
                api.Params(k_eps=1e-4), api.Params(k_eps=0.0, h=0.5),
                api.Params(nbr_c=0.25), api.Params(nbr_c=0.0, h=2.0),
                api.Params(nbr_c=0.25, si_scale=1)):
        out, ref = _run(A, "f32", "f32", prm)
        parity.compare(out, ref, "f32")


def test_fwd_clamp_float():
    A = scenes.planar(scenes.pixel_art(48, 260, scenes.seed_for(4, 3))) / 255.0
    out, ref = _run(A, "u8", "f32", api.Params(clamp_float=True))
    parity.compare(out, ref, "f32", clamp_float=True)


def test_fwd_analytic_step_64():
    """64x64 sin(2 pi x) cos(3 pi y) + step, h = 1/64 (pixel centres)."""
    A = scenes.analytic_step(64)[None]
    for mode in (0, 1):
        out, ref = _run(A, "f32", "f32", api.Params(h=1 / 64, out_mode=mode))
        parity.compare(out, ref, "f32", value_range=float(A.max() - A.min()))


@pytest.mark.parametrize("layout", ["hwc"])
def test_fwd_interleaved_layout(layout):
    img = scenes.piecewise_smooth(41, 333, seed=scenes.seed_for(2, 5), scale_features=True)
    A = scenes.planar(img) / 255.0
    out, ref = _run(A, "u8", "u8", layout=layout)
    parity.compare(out, ref, "u8")


def test_fwd_strided_views_and_batch():
    base = torch.rand(3, 90, 700, device=DEV)
    view = base[:, 5:77, 11:612]  # cropped, non-contiguous rows
    out_full = torch.zeros(3, 200, 1400, device=DEV)
    out_view = out_full[:, 3:147, 7:1209]
    api.zoom2x_fwd(view, out=out_view)
    torch.cuda.synchronize()
    ref = parity.oracle_planes(view.double().cpu().numpy(), api.Params())
    parity.compare(out_view, ref, "f32")
    # untouched margin stays zero
    assert float(out_full[:, :3].abs().max()) == 0.0
    assert float(out_full[:, :, :7].abs().max()) == 0.0
    # NCHW batch folds into planes
    xb = torch.rand(4, 2, 19, 250, device=DEV)
    ob = api.zoom2x_fwd(xb)
    torch.cuda.synchronize()
    refb = parity.oracle_planes(xb.double().cpu().numpy(), api.Params())
    parity.compare(ob, refb, "f32")


def test_fwd_tile_shape_invariance():
    """Every value is formed by the same arithmetic whatever the band height,
    so outputs are bit-identical across tile shapes."""
    x = torch.rand(2, 301, 517, device=DEV)
    outs = [api.zoom2x_fwd(x, rows_per_tile=r) for r in (0, 1, 7, 64, 100, 400)]
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


def _windows(H, W, count, size=(24, 40), margin=6):
    wins = [(0, 0), (0, W - size[1]), (H - size[0], 0), (H - size[0], W - size[1])]
    for _ in range(count):
        wins.append((int(RNG.integers(0, H - size[0] + 1)), int(RNG.integers(0, W - size[1] + 1))))
    return wins


def _check_windows(A01, out_gpu, dt, params, wins, size=(24, 40), margin=6):
    """Oracle on input crops with a margin: output quads whose footprint
    (-4..+5 input cells) stays inside the crop equal the full-image result;
    at the image border the crop reaches the border, so clamping agrees."""
    C, H, W = A01.shape
    ties = 0
    for (r0, c0) in wins:
        ra, rb = max(0, r0 - margin), min(H, r0 + size[0] + margin)
        ca, cb = max(0, c0 - margin), min(W, c0 + size[1] + margin)
        ref = parity.oracle_planes(A01[:, ra:rb, ca:cb], params)
        pr, pc = 2 * (r0 - ra), 2 * (c0 - ca)
        ref = ref[:, pr:pr + 2 * size[0], pc:pc + 2 * size[1]]
        g = out_gpu[:, 2 * r0:2 * r0 + 2 * size[0], 2 * c0:2 * c0 + 2 * size[1]]
        ties += parity.compare(g, ref, dt)[1]
    return ties


def test_fwd_full_hd_rgb_u8_sampled():
    """1920x1080 RGB uint8 piecewise-smooth scene -> 3840x2160, launched as
    the benchmark launches it; the oracle checks sampled windows (corners
    included)."""
    img = scenes.piecewise_smooth(1080, 1920, seed=scenes.seed_for(2))
    x = torch.from_numpy(scenes.planar(img)).to(DEV)
    out = api.zoom2x_fwd(x).cpu()
    A01 = scenes.planar(img).astype(np.float64) / 255.0
    ties = _check_windows(A01, out, "u8", api.Params(), _windows(1080, 1920, 12))
    assert ties < 20


def test_fwd_4k_precision_sweep_sampled():
    """3840x2160 RGB scene stored as uint8 / FP16 / BF16 / FP32 -> 7680x4320."""
    img = scenes.piecewise_smooth(2160, 3840, seed=scenes.seed_for(4))
    A01 = scenes.planar(img).astype(np.float64) / 255.0
    wins = _windows(2160, 3840, 4)
    for dt in ("u8", "f16", "bf16", "f32"):
        x = parity.encode(A01, dt).to(DEV)
        out = api.zoom2x_fwd(x).cpu()
        _check_windows(parity.decode(x.cpu()), out, dt, api.Params(), wins)


@pytest.mark.parametrize("n,m", [(16384, 16384), (16000, 16001)])
def test_fwd_large_planes_64bit_offsets(n, m):
    """3 x n x m uint8 input: output offsets exceed 2^31; the odd width puts
    the rows at every byte alignment."""
    x = torch.empty(3, n, m, dtype=torch.uint8, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(7)
    x.copy_(torch.randint(0, 256, (3, n, m), device=DEV, generator=g, dtype=torch.uint8))
    out = api.zoom2x_fwd(x)
    torch.cuda.synchronize()
    A01 = x[:, -40:, -60:].cpu().numpy().astype(np.float64) / 255.0
    ref = parity.oracle_planes(A01, api.Params())
    # bottom-right corner of the last plane: the largest output offsets
    parity.compare(out[:, -2 * 30:, -2 * 50:].cpu(), ref[:, -60:, -100:], "u8")
    del out, x
    torch.cuda.empty_cache()


# Widths that keep every row 16-byte aligned (full vector stores of the
# output rows at every storage type).
ALIGNED = [(1, 16), (5, 32), (37, 496), (70, 512), (9, 1024), (130, 256)]


@pytest.mark.parametrize("shape", ALIGNED)
@pytest.mark.parametrize("dt", DTS)
@pytest.mark.parametrize("mode", [0, 1])
def test_fwd_aligned_rows(shape, dt, mode):
    A = RNG.random((3,) + shape)
    out, ref = _run(A, dt, dt, api.Params(out_mode=mode))
    parity.compare(out, ref, dt)


@pytest.mark.parametrize("in_dt", DTS)
@pytest.mark.parametrize("out_dt", DTS)
def test_fwd_aligned_storage_pairs(in_dt, out_dt):
    img = scenes.piecewise_smooth(37, 512, seed=scenes.seed_for(4, 8), scale_features=True)
    A = scenes.planar(img).astype(np.float64) / 255.0
    out, ref = _run(A, in_dt, out_dt)
    parity.compare(out, ref, out_dt)


def _strided_copy(xs):
    """The same values with column stride 2."""
    wide = torch.zeros(xs.shape[:-1] + (2 * xs.shape[-1],), device=DEV, dtype=xs.dtype)
    wide[..., ::2] = xs
    return wide[..., ::2]


def test_fwd_unit_and_strided_columns_agree_bitwise():
    """The same values at unit column stride and at column stride 2 give
    bit-identical outputs for every band height, for 16-byte aligned rows
    (width 512) and for rows at every alignment (width 513, padded rows)."""
    x = torch.rand(2, 203, 513, device=DEV)
    for dt in (torch.uint8, torch.float16, torch.bfloat16):
        xs = (x * 255).to(torch.uint8) if dt == torch.uint8 else x.to(dt)
        for img in (xs[:, :, :512].contiguous(), xs, xs[:, :, :511]):
            xv = _strided_copy(img)
            for r in (0, 1, 7, 64, 100):
                a = api.zoom2x_fwd(img, rows_per_tile=r)
                b = api.zoom2x_fwd(xv, rows_per_tile=r)
                torch.cuda.synchronize()
                assert torch.equal(a, b), (dt, tuple(img.shape), img.stride(), r)


@pytest.mark.parametrize("dt", ["u8", "f16", "bf16"])
def test_fwd_unaligned_rows_and_views(dt):
    """Rows that start anywhere: odd widths, a crop that starts at an odd
    element of an odd row, and single columns; parity with the oracle."""
    for shape in [(3, 1), (7, 13), (41, 257), (33, 499), (19, 771)]:
        A = RNG.random((2,) + shape)
        out, ref = _run(A, dt, dt)
        parity.compare(out, ref, dt)
    big = RNG.random((2, 61, 530))
    xb = parity.encode(big, dt).to(DEV)
    view = xb[:, 3:58, 5:522]  # base, rows and planes all off 16-byte boundaries
    out = api.zoom2x_fwd(view)
    torch.cuda.synchronize()
    ref = parity.oracle_planes(parity.decode(view.cpu()), api.Params())
    parity.compare(out, ref, dt)


def test_fwd_no_abandoned_waits():
    from paper_2312_00229_gb300 import binding as B
    B.weno_wait_timeouts(reset=True)
    x = torch.rand(3, 300, 1024, device=DEV)
    for r in (0, 16, 128):
        api.zoom2x_fwd(x, rows_per_tile=r)
    api.zoom2x_fwd((x * 255).to(torch.uint8))
    torch.cuda.synchronize()
    assert B.weno_wait_timeouts() == 0


def test_fwd_weight_forms_at_the_range_limits():
    """beta = 2 weights are taken as 1/D^2 directly when the input type bounds
    the data (uint8, FP16) and the eps / h setting keeps every weight in the
    FP32 range, else in the scale-free form (D_min/D)^2.  Parity on both
    sides of that choice: FP16 data at the ends of its range, a vanishing
    eps_h (tiny k_eps or h) and a huge neighbour weight (large h)."""
    big = scenes.planar(scenes.piecewise_smooth(31, 260, seed=scenes.seed_for(4, 9),
                                                scale_features=True)).astype(np.float64)
    big = (big / 255.0 * 2.0 - 1.0) * 65504.0  # FP16 range, both signs
    big[0, 3, 10:20] = 65504.0
    big[1, 7, 40:44] = -65504.0
    x = torch.from_numpy(big.astype(np.float16))
    for prm in (api.Params(), api.Params(si_scale=1), api.Params(h=1e4)):
        out = api.zoom2x_fwd(x.to(DEV), prm, out_dtype=torch.float32)
        torch.cuda.synchronize()
        ref = parity.oracle_planes(x.double().numpy(), prm)
        parity.compare(out, ref, "f32", value_range=float(ref.max() - ref.min()))
    A = scenes.planar(scenes.pixel_art(40, 250, scenes.seed_for(4, 10))) / 255.0
    for prm in (api.Params(k_eps=1e-30), api.Params(h=1e-6), api.Params(h=1e4),
                api.Params(h=1e-6, k_eps=1e6)):
        for in_dt in ("u8", "f16"):
            out, ref = _run(A, in_dt, "f32", prm)
            parity.compare(out, ref, "f32")


def test_fwd_direct_and_scale_free_weights_agree():
    """The same FP16 values zoomed from FP16 storage (direct 1/D^2 weights)
    and from FP32 storage (scale-free weights, the type does not bound the
    data) agree to a few FP32 rounding steps."""
    x = torch.rand(3, 77, 300, device=DEV).to(torch.float16)
    a = api.zoom2x_fwd(x, out_dtype=torch.float32)
    b = api.zoom2x_fwd(x.float(), out_dtype=torch.float32)
    torch.cuda.synchronize()
    assert (a - b).abs().max().item() <= 4e-6


def test_fwd_data_bound_selects_direct_weights():
    """FP32 data with a caller-given bound take the direct 1/D^2 weights:
    parity with the oracle, agreement with the scale-free weights (no bound)
    to a few FP32 rounding steps, and a bound too large for the range proof
    (1e30) falls back to the scale-free form with the same parity."""
    A = RNG.random((2, 53, 301))
    for bound in (1.0, 7.5, 1e30):
        out, ref = _run(A, "f32", "f32", api.Params(data_bound=bound))
        parity.compare(out, ref, "f32")
    x = torch.from_numpy(A.astype(np.float32)).to(DEV)
    a = api.zoom2x_fwd(x, api.Params(data_bound=1.0))
    b = api.zoom2x_fwd(x)
    torch.cuda.synchronize()
    assert (a - b).abs().max().item() <= 4e-6
    big = torch.from_numpy((A * 2e3 - 1e3).astype(np.float32))
    out = api.zoom2x_fwd(big.to(DEV), api.Params(data_bound=1e3))
    torch.cuda.synchronize()
    ref = parity.oracle_planes(big.double().numpy(), api.Params())
    parity.compare(out, ref, "f32", value_range=float(ref.max() - ref.min()))


@pytest.mark.parametrize("dt", ["u8", "f16", "f32"])
@pytest.mark.parametrize("mode", [0, 1])
def test_fwd_narrow_and_wide_ctas_agree_bitwise(dt, mode):
    """128-thread CTAs (119-column strips) and 256-thread CTAs (247-column
    strips) give the same outputs bit for bit at widths that end their last
    strip anywhere, and the narrow form matches the oracle."""
    p = api.Params(out_mode=mode)
    for shape in [(9, 1), (13, 118), (21, 119), (17, 120), (40, 247), (37, 512), (6, 1001)]:
        A = RNG.random((2,) + shape)
        x = parity.encode(A, dt).to(DEV)
        a = api.zoom2x_fwd(x, p, tile_width=119)
        b = api.zoom2x_fwd(x, p, tile_width=247)
        c = api.zoom2x_fwd(x, p)  # the library's choice
        torch.cuda.synchronize()
        assert torch.equal(a, b) and torch.equal(a, c), (dt, mode, shape)
    ref = parity.oracle_planes(parity.decode(x.cpu()), p)
    parity.compare(a.cpu(), ref, dt)


@pytest.mark.parametrize("dt", ["u8", "f16", "bf16", "f32"])
@pytest.mark.parametrize("mode", [0, 1])
def test_fwd_paired_columns_agree_bitwise(dt, mode):
    """Two coarse columns per thread (tile widths 246 and 118: 128 and 64
    threads) form every value by the same expressions as one column per
    thread, so the outputs agree bit for bit; widths end the last strip
    anywhere, odd widths leave one column of a pair idle, and 2n-1 mode
    drops the last fine column of a quad."""
    p = api.Params(out_mode=mode)
    shapes = [(9, 1), (5, 2), (13, 117), (21, 118), (17, 119), (11, 245), (40, 246),
              (23, 247), (37, 512), (6, 1001)]
    for shape in shapes:
        A = RNG.random((2,) + shape)
        x = parity.encode(A, dt).to(DEV)
        ref1 = api.zoom2x_fwd(x, p, tile_width=247)
        for tw in (246, 118):
            got = api.zoom2x_fwd(x, p, tile_width=tw)
            torch.cuda.synchronize()
            assert torch.equal(got, ref1), (dt, mode, shape, tw)


def test_fwd_paired_columns_strided_views():
    """Output rows not aligned to four elements (a column-cropped view) take
    the per-element stores of the paired tile."""
    A = RNG.random((3, 30, 77))
    x = parity.encode(A, "u8").to(DEV)
    big = torch.full((3, 60, 160), 7, dtype=torch.uint8, device=DEV)
    view = big[:, :, 1:155]
    api.zoom2x_fwd(x, out=view, tile_width=246)
    ref = api.zoom2x_fwd(x, tile_width=247)
    torch.cuda.synchronize()
    assert torch.equal(view, ref)
    assert torch.all(big[:, :, 0] == 7) and torch.all(big[:, :, 155:] == 7)


def test_fwd_rejects_other_tile_widths():
    from paper_2312_00229_gb300 import binding as B
    x = torch.zeros(3, 8, 8, dtype=torch.uint8, device=DEV)
    o = torch.zeros(3, 16, 16, dtype=torch.uint8, device=DEV)
    for tw in (1, 117, 120, 245, 248, 256, -1):
        rc = B.weno_zoom2x_fwd_tiled(api.image(x), 0, api.image(o), 0, api.Params().c(), 0, tw,
                                     api._stream(x.device))
        assert rc == B.WENO_EINVAL, tw
