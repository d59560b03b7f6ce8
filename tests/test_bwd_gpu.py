"""Adjoint parity: GPU input gradient (through the C ABI) against the FP64
reference gradient (autograd of the independent float64 restatement in
``oracle/wdweno_torch.py``) and FP64 central differences of the C oracle.

Tolerance: max |g_gpu - g_ref| <= GRAD_TOL x max |g_ref| (derivation in the
design notes: FP32 rounding of differences of O(1) pixel values, amplified
by at most the (p - u) / D factor of the weight derivative)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle import wdweno_torch as wt
from paper_2312_00229_gb300 import api, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"
RNG = np.random.default_rng(99)
GRAD_TOL = 2e-4


def _ref_grad(A: np.ndarray, G: np.ndarray, params: api.Params) -> np.ndarray:
    At = torch.from_numpy(A.copy()).requires_grad_(True)
    U = wt.zoom2x(At, beta=params.beta, k_eps=params.k_eps, h=params.h,
                  si_scale=params.si_scale, out_mode=params.out_mode,
                  nbr_c=(params.nbr_c, params.nbr_c))
    (g,) = torch.autograd.grad((U * torch.from_numpy(G)).sum(), At)
    return g.numpy()


def _gpu_grad(A: np.ndarray, G: np.ndarray, params: api.Params) -> np.ndarray:
    x = torch.from_numpy(A.astype(np.float32)).to(DEV)
    g = torch.from_numpy(G.astype(np.float32)).to(DEV)
    gi = api.zoom2x_bwd(x, g, params)
    torch.cuda.synchronize()
    return gi.double().cpu().numpy()


def _check(A, G, params):
    # the reference differentiates at the FP32-rounded input the GPU sees
    A = A.astype(np.float32).astype(np.float64)
    ref = _ref_grad(A, G, params)
    got = _gpu_grad(A, G, params)
    scale = max(np.abs(ref).max(), 1e-30)
    err = np.abs(got - ref).max() / scale
    assert err <= GRAD_TOL, err
    return err


@pytest.mark.parametrize("shape", [(1, 1), (1, 6), (5, 1), (2, 3), (7, 9), (16, 16), (23, 41)])
@pytest.mark.parametrize("mode", [0, 1])
def test_bwd_random(shape, mode):
    params = api.Params(out_mode=mode)
    A = RNG.random((2,) + shape)
    oh, ow = api.out_hw(shape[0], shape[1], params)
    G = RNG.normal(size=(2, oh, ow))
    _check(A, G, params)


@pytest.mark.parametrize("beta", [0.0, 0.1, 1.0, 3.0])
def test_bwd_beta(beta):
    params = api.Params(beta=beta)
    A = RNG.random((1, 12, 17))
    G = RNG.normal(size=(1, 24, 34))
    _check(A, G, params)


def test_bwd_params():
    A = RNG.random((1, 11, 13))
    G = RNG.normal(size=(1, 22, 26))
    for params in (api.Params(si_scale=1), api.Params(h=0.25), api.Params(k_eps=1e-3),
                   api.Params(nbr_c=0.25), api.Params(nbr_c=0.5, h=2.0)):
        _check(A, G, params)


def test_bwd_scene_crop():
    img = scenes.piecewise_smooth(48, 64, seed=scenes.seed_for(5, 1), scale_features=True)
    A = scenes.planar(img).astype(np.float64) / 255.0
    G = RNG.normal(size=(3, 96, 128))
    _check(A, G, api.Params())


def test_bwd_matches_central_differences():
    """FP64 central differences (step 1e-6) of the C oracle on a 16x16 crop."""
    n = 16
    A = RNG.random((n, n)).astype(np.float32).astype(np.float64)
    G = RNG.normal(size=(2 * n, 2 * n))
    got = _gpu_grad(A[None], G[None], api.Params())[0]
    scale = np.abs(got).max()
    for (i, j) in [(0, 0), (3, 9), (8, 8), (15, 0), (15, 15), (6, 14)]:
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += 1e-6
        Am[i, j] -= 1e-6
        fd = ((oracle.zoom2x(Ap) * G).sum() - (oracle.zoom2x(Am) * G).sum()) / 2e-6
        assert abs(got[i, j] - fd) <= GRAD_TOL * scale, (i, j, got[i, j], fd)


def test_autograd_function_and_batch():
    x = torch.rand(2, 3, 20, 31, device=DEV, requires_grad=True)
    y = api.zoom2x(x)
    w = torch.randn_like(y)
    (y * w).sum().backward()
    ref = _ref_grad(x.detach().double().cpu().numpy().reshape(6, 20, 31),
                    w.double().cpu().numpy().reshape(6, 40, 62), api.Params())
    got = x.grad.double().cpu().numpy().reshape(6, 20, 31)
    assert np.abs(got - ref).max() <= GRAD_TOL * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(130, 300), (300, 40), (61, 250)])
def test_bwd_several_strips_and_bands(shape):
    """Sizes that span several column strips and row bands of both adjoint
    sweeps, with ragged last strips and bands."""
    A = RNG.random((1,) + shape)
    G = RNG.normal(size=(1, 2 * shape[0], 2 * shape[1]))
    _check(A, G, api.Params())


@pytest.mark.parametrize("n", [14, 27, 33, 45, 58])
def test_bwd_band_step_forms(n):
    """Heights whose bands start at different rows modulo 4, so that the
    sweeps switch between their guarded steps and their four-step groups of
    guard-free steps at every alignment, and bands too short for any group."""
    A = RNG.random((3, n, 70))
    G = RNG.normal(size=(3, 2 * n, 140))
    _check(A, G, api.Params())


def test_bwd_windowed_at_bench_size():
    """32x3x512x512 planes (the fwd+bwd workload) with grad_out nonzero only in
    a 24x24 window of one plane: the gradient is compared with the FP64
    reference gradient of a crop that holds the window's whole footprint,
    and must vanish outside it in every plane."""
    rng = np.random.default_rng(7)
    img = scenes.piecewise_smooth(512, 512, seed=scenes.seed_for(5, 3), scale_features=True)
    A = scenes.planar(img).astype(np.float32) / np.float32(255.0)
    x = torch.from_numpy(np.broadcast_to(A, (32, 3, 512, 512)).copy()).to(DEV)
    g = torch.zeros(32, 3, 1024, 1024, device=DEV)
    P0, Q0 = 601, 333  # odd offsets: the window starts on an x / S row and an E column
    win = rng.normal(size=(24, 24)).astype(np.float32)
    g[17, 1, P0:P0 + 24, Q0:Q0 + 24] = torch.from_numpy(win).to(DEV)
    gi = api.zoom2x_bwd(x, g).double().cpu().numpy()
    # crop: the quads of the window with a 16-cell margin (footprint: 5 cells)
    i0, j0 = P0 // 2 - 16, Q0 // 2 - 16
    i1, j1 = (P0 + 24) // 2 + 16, (Q0 + 24) // 2 + 16
    Ac = A[1, i0:i1, j0:j1].astype(np.float64)[None]
    Gc = np.zeros((1, 2 * (i1 - i0), 2 * (j1 - j0)))
    Gc[0, P0 - 2 * i0:P0 - 2 * i0 + 24, Q0 - 2 * j0:Q0 - 2 * j0 + 24] = win
    ref = _ref_grad(Ac, Gc, api.Params())[0]
    got = gi[17, 1, i0:i1, j0:j1]
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(got - ref).max() <= GRAD_TOL * scale
    outside = gi.copy()
    outside[17, 1, i0:i1, j0:j1] = 0.0
    assert not np.any(outside)


def test_bwd_writes_only_grad_in():
    """grad_in placed inside a poisoned buffer (guard bands before, after and
    between rows): the adjoint writes exactly the grad_in elements."""
    A = RNG.random((2, 37, 53)).astype(np.float32)
    G = RNG.normal(size=(2, 74, 106)).astype(np.float32)
    x = torch.from_numpy(A).to(DEV)
    g = torch.from_numpy(G).to(DEV)
    poison = -7.25e30
    big = torch.full((2, 37 + 8, 53 + 24), poison, device=DEV)
    gin = big[:, 4:41, 9:62]  # row stride 77, channel stride 45 * 77
    need = api.B.weno_zoom2x_bwd_workspace_bytes(api.image(x))
    ws = torch.empty(need, dtype=torch.uint8, device=DEV)
    rc = api.B.weno_zoom2x_bwd(api.image(x), api.image(g), api.image(gin), api.Params().c(),
                               ctypes.c_void_p(ws.data_ptr()), need, api._stream(x.device))
    api.B.check("weno_zoom2x_bwd", rc)
    torch.cuda.synchronize()
    ref = api.zoom2x_bwd(x, g)
    assert torch.equal(gin, ref)
    mask = torch.ones_like(big, dtype=torch.bool)
    mask[:, 4:41, 9:62] = False
    assert torch.all(big[mask] == poison)
