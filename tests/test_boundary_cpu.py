"""C-ABI boundary checks that need no GPU: the library builds and loads,
exports every entry point ``include/wdweno.h`` declares, and rejects bad
arguments on the host before any launch."""
import ctypes
import os
import re

import pytest
import torch

from paper_2312_00229_gb300 import binding as B
from paper_2312_00229_gb300 import api

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "wdweno.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(weno_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_match_binding():
    assert _declared() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = B.load()
    for name in _declared():
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_params_default():
    p = B.weno_params_default()
    assert (p.beta, p.k_eps, p.h, p.si_scale, p.out_mode, p.clamp_float, p.data_bound,
            p.nbr_c) == (pytest.approx(2.0), pytest.approx(1e-8), pytest.approx(1.0), 0, 0, 0,
                         0.0, 0.125)


def test_status_strings():
    for st in (0, -1, -2, -3, -4, -5, -99):
        assert isinstance(B.weno_status_string(st), str) and B.weno_status_string(st)


def _img(ptr, h, w, c, sc=None, sh=None, sw=1):
    im = B.weno_image()
    im.data = ptr
    im.height, im.width, im.channels = h, w, c
    im.stride_w = sw
    im.stride_h = sh if sh is not None else w * sw
    im.stride_c = sc if sc is not None else h * im.stride_h
    return im


FAKE_IN = 0x10000000
FAKE_OUT = 0x20000000


def test_fwd_rejects_bad_arguments_without_launching():
    p = B.weno_params_default()
    good_in = _img(FAKE_IN, 4, 5, 3)
    good_out = _img(FAKE_OUT, 8, 10, 3)
    cases = [
        (_img(0, 4, 5, 3), good_out, B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),        # null
        (_img(FAKE_IN, 0, 5, 3), good_out, B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),  # empty
        (_img(FAKE_IN, 4, 5, 3, sw=0), good_out, B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),
        (good_in, _img(FAKE_OUT, 8, 9, 3), B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),  # shape
        (good_in, _img(FAKE_OUT, 8, 10, 2), B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),  # channels
        (good_in, good_out, 7, B.WENO_U8, B.WENO_EDTYPE),
        (good_in, good_out, B.WENO_U8, -1, B.WENO_EDTYPE),
        (good_in, _img(FAKE_IN + 10, 8, 10, 3), B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),  # overlap
    ]
    for i, (a, b, ta, tb, want) in enumerate(cases):
        assert B.weno_zoom2x_fwd(a, ta, b, tb, p, None) == want, i
    bad = B.weno_params_default()
    bad.h = 0.0
    assert B.weno_zoom2x_fwd(good_in, 0, good_out, 0, bad, None) == B.WENO_EINVAL
    bad = B.weno_params_default()
    bad.beta = -1.0
    assert B.weno_zoom2x_fwd(good_in, 0, good_out, 0, bad, None) == B.WENO_EINVAL
    bad = B.weno_params_default()
    bad.out_mode = 5
    assert B.weno_zoom2x_fwd(good_in, 0, good_out, 0, bad, None) == B.WENO_EINVAL
    for v in (-1.0, float("inf"), float("nan")):  # data_bound must be finite and >= 0
        bad = B.weno_params_default()
        bad.data_bound = v
        assert B.weno_zoom2x_fwd(good_in, 0, good_out, 0, bad, None) == B.WENO_EINVAL
    for v in (-0.125, float("inf"), float("nan")):  # nbr_c must be finite and >= 0
        bad = B.weno_params_default()
        bad.nbr_c = v
        assert B.weno_zoom2x_fwd(good_in, 0, good_out, 0, bad, None) == B.WENO_EINVAL
    # (2n-1) mode changes the expected output shape
    m1 = B.weno_params_default()
    m1.out_mode = 1
    assert B.weno_zoom2x_fwd(good_in, 0, good_out, 0, m1, None) == B.WENO_EINVAL
    # unsupported tile shapes: band heights outside 0..4096, widths other than
    # 0 (the library's choice), 247 (256-thread CTAs) and 119 (128 threads)
    assert B.weno_zoom2x_fwd_tiled(good_in, 0, good_out, 0, p, -1, 0, None) == B.WENO_EINVAL
    assert B.weno_zoom2x_fwd_tiled(good_in, 0, good_out, 0, p, 4097, 0, None) == B.WENO_EINVAL
    for tw in (-1, 1, 100, 117, 120, 128, 245, 248, 256):
        assert B.weno_zoom2x_fwd_tiled(good_in, 0, good_out, 0, p, 0, tw, None) == B.WENO_EINVAL


def test_bwd_rejects_bad_arguments_without_launching():
    p = B.weno_params_default()
    x = _img(FAKE_IN, 4, 5, 1)
    go = _img(FAKE_OUT, 8, 10, 1)
    gi = _img(0x30000000, 4, 5, 1)
    need = B.weno_zoom2x_bwd_workspace_bytes(x)
    assert need == 4 * 2 * (4 + 4) * (5 + 4)  # X_bar and partial A_bar, 2 ghost cells a side
    assert B.weno_zoom2x_bwd(x, go, gi, p, None, need, None) == B.WENO_EWORKSPACE
    assert B.weno_zoom2x_bwd(x, go, gi, p, 0x40000000, need - 1, None) == B.WENO_EWORKSPACE
    assert B.weno_zoom2x_bwd(x, go, gi, p, 0x40000004, need, None) == B.WENO_EWORKSPACE
    assert B.weno_zoom2x_bwd(x, go, _img(0x30000000, 4, 4, 1), p, 0x40000000, need,
                             None) == B.WENO_EINVAL
    assert B.weno_zoom2x_bwd(x, go, _img(FAKE_IN, 4, 5, 1), p, 0x40000000, need,
                             None) == B.WENO_EINVAL  # grad_in aliases x
    assert B.weno_zoom2x_bwd_workspace_bytes(_img(FAKE_IN, 0, 5, 1)) == 0



def test_batched_rejects_bad_arguments_without_launching():
    p = B.weno_params_default()
    need = B.weno_zoom2x_batched_workspace_bytes(3)
    assert need >= 16 + 8 * 4 and need % 16 == 0  # head, total, count + 1 prefixes
    assert B.weno_zoom2x_batched(0, None, 0, None, 0, p, None, 0, 0, 0, None) == B.WENO_OK
    assert B.weno_zoom2x_batched(-1, 1, 0, 1, 0, p, 2, need, 0, 0, None) == B.WENO_EINVAL
    assert B.weno_zoom2x_batched(3, None, 0, 1, 0, p, 2, need, 0, 0, None) == B.WENO_EINVAL
    assert B.weno_zoom2x_batched(3, 1, 9, 1, 0, p, 2, need, 0, 0, None) == B.WENO_EDTYPE
    assert B.weno_zoom2x_batched(3, 1, 0, 1, 0, p, None, need, 0, 0, None) == B.WENO_EWORKSPACE
    assert B.weno_zoom2x_batched(3, 1, 0, 1, 0, p, 0x100, need - 16, 0, 0,
                                 None) == B.WENO_EWORKSPACE
    for tw in (-1, 1, 77, 117, 120, 128, 245, 248, 256):  # widths other than 0, 247, 119, 246, 118
        assert B.weno_zoom2x_batched(3, 1, 0, 1, 0, p, 0x100, need, 0, tw,
                                     None) == B.WENO_EINVAL
    assert B.weno_zoom2x_batched(3, 1, 0, 1, 0, p, 0x100, need, 4097, 0, None) == B.WENO_EINVAL


def test_descriptor_folding_on_host_tensors():
    """Descriptor construction (pure host logic) for the layouts the API takes."""
    x = torch.zeros(3, 7, 9)
    im = api.image(x)
    assert (im.height, im.width, im.channels, im.stride_c, im.stride_h, im.stride_w) == (
        7, 9, 3, 63, 9, 1)
    x = torch.zeros(7, 9, 4)
    im = api.image(x, "hwc")
    assert (im.height, im.width, im.channels, im.stride_c, im.stride_h, im.stride_w) == (
        7, 9, 4, 1, 36, 4)
    x = torch.zeros(5, 3, 7, 9)
    im = api.image(x)
    assert (im.height, im.width, im.channels, im.stride_c) == (7, 9, 15, 63)
    x = torch.zeros(3, 20, 30)[:, 2:9, 5:14]  # cropped view
    im = api.image(x)
    assert (im.height, im.width, im.channels, im.stride_c, im.stride_h, im.stride_w) == (
        7, 9, 3, 600, 30, 1)
    with pytest.raises(ValueError):
        api.image(torch.zeros(4, 3, 8, 8).transpose(0, 1))
    assert api.out_hw(7, 9, api.Params()) == (14, 18)
    assert api.out_hw(7, 9, api.Params(out_mode=1)) == (13, 17)


def test_api_refuses_cpu_tensors():
    with pytest.raises(ValueError):
        api.zoom2x_fwd(torch.zeros(1, 4, 4))


def test_resample_rejects_bad_arguments_without_launching():
    p = B.weno_params_default()
    good_in = _img(FAKE_IN, 4, 5, 3)
    good_out = _img(FAKE_OUT, 11, 2, 3)
    cases = [
        (_img(0, 4, 5, 3), good_out, B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),        # null
        (good_in, _img(FAKE_OUT, 0, 2, 3), B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),  # empty out
        (good_in, _img(FAKE_OUT, 11, 2, 2), B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),  # channels
        (good_in, good_out, 9, B.WENO_U8, B.WENO_EDTYPE),
        (good_in, _img(FAKE_IN + 3, 11, 2, 3), B.WENO_U8, B.WENO_U8, B.WENO_EINVAL),  # overlap
        (_img(FAKE_IN, 4, 5, 70000), _img(FAKE_OUT, 6, 6, 70000), B.WENO_U8, B.WENO_U8,
         B.WENO_EINVAL),  # channels < 65536
        (good_in, _img(FAKE_OUT, 600000, 2, 3), B.WENO_U8, B.WENO_U8, B.WENO_ERANGE),
    ]
    for i, (a, b, ta, tb, want) in enumerate(cases):
        assert B.weno_resample(a, ta, b, tb, p, None) == want, i
    bad = B.weno_params_default()
    bad.beta = float("nan")
    assert B.weno_resample(good_in, 0, good_out, 0, bad, None) == B.WENO_EINVAL


def test_api_zoom_levels_and_cpu_refusal():
    assert api.zoom_levels(1080, 1920, 3240, 5760) == 2
    assert api.zoom_levels(5, 5, 4, 4) == 0
    with pytest.raises(ValueError):
        api.resample(torch.zeros(1, 4, 4), 8, 8)
    with pytest.raises(ValueError):
        api.zoom_to(torch.zeros(1, 4, 4), 8, 8)


def test_package_exports_resolve():
    import paper_2312_00229_gb300 as pkg
    for name in pkg.__all__:
        assert getattr(pkg, name) is not None, name


def test_fp32_probe_rejects_bad_arguments_and_counts_ops():
    assert B.weno_fp32_probe(0, 1, 0x100, None) == B.WENO_EINVAL
    assert B.weno_fp32_probe(1, 0, 0x100, None) == B.WENO_EINVAL
    assert B.weno_fp32_probe(1, 1, None, None) == B.WENO_EINVAL
    # 256 threads x 8 rounds x 16 chains per iteration
    assert B.weno_fp32_probe_ops(3, 5) == 3 * 256 * 5 * 8 * 16
    assert B.weno_fp32_probe(1 << 25, 1, 0x100, None) == B.WENO_EINVAL
    assert B.weno_fp32_probe_ops(1, 1 << 25) == -1 and B.weno_fp32_probe_ops(0, 1) == -1
