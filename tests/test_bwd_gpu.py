"""Adjoint parity: GPU input gradient (through the C ABI) against the FP64
reference gradient (autograd of the independent float64 restatement in
``oracle/wdweno_torch.py``) and FP64 central differences of the C oracle.

Tolerance: max |g_gpu - g_ref| <= GRAD_TOL x max |g_ref| (derivation in the
design notes: FP32 rounding of differences of O(1) pixel values, amplified
by at most the (p - u) / D factor of the weight derivative)."""
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
