"""The batched entry point that allocates nothing (weno_zoom2x_batched_noalloc).

Callers that cannot allocate device memory (a real-time pipeline where
cudaMalloc could stall other streams, or a plugin handed only pointers) use
this variant; its tile queue lives in a fixed array inside the library.  Its
output must equal the workspace-taking batched entry point's, and the shared
array must not carry state from one call into the next, so the check runs on
two consecutive calls with different images.  Kept in its own file so that
pytest collects it last."""
import ctypes

import pytest
import torch

from paper_2312_00229_gb300 import api
from paper_2312_00229_gb300 import binding as B

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _batch(seed, sizes):
    g = torch.Generator(device=DEV).manual_seed(seed)
    return [torch.randint(0, 256, (3, h, w), device=DEV, generator=g, dtype=torch.uint8)
            for (h, w) in sizes]


def _noalloc(plan):
    rc = B.weno_zoom2x_batched_noalloc(plan.count, ctypes.c_void_p(plan.d_in.data_ptr()),
                                       plan.in_t, ctypes.c_void_p(plan.d_out.data_ptr()),
                                       plan.out_t, plan.params.c(), 0, 0,
                                       api._stream(plan.device))
    B.check("weno_zoom2x_batched_noalloc", rc)


def test_noalloc_matches_batched_on_two_calls():
    sizes = [[(1, 1), (40, 300), (257, 93), (64, 64)], [(500, 700), (3, 5), (97, 1024)]]
    for call, sz in enumerate(sizes):
        imgs = _batch(100 + call, sz)
        plan = api.BatchedPlan(imgs)
        for o in plan.outputs:
            o.fill_(7)
        _noalloc(plan)
        got = [o.clone() for o in plan.outputs]
        ref = api.zoom2x_batched(imgs)  # workspace-taking entry point
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b)


def test_noalloc_at_the_image_limit():
    # Exactly WENO_NOALLOC_MAX_IMAGES images fill the array to its bound: the
    # call must succeed and match the workspace-taking batched call.  1x1 and
    # 2x3 images keep it small.
    n = B.WENO_NOALLOC_MAX_IMAGES
    sizes = [(1, 1) if i % 2 else (2, 3) for i in range(n)]
    imgs = _batch(7, sizes)
    plan = api.BatchedPlan(imgs, rows_per_tile=16)
    for o in plan.outputs:
        o.fill_(7)
    _noalloc(plan)
    got = torch.cat([o.flatten() for o in plan.outputs])
    ref = api.BatchedPlan(imgs, rows_per_tile=16).run()
    torch.cuda.synchronize()
    assert torch.equal(got, torch.cat([o.flatten() for o in ref]))


def test_noalloc_rejects_too_many_images():
    p = B.weno_params_default()
    rc = B.weno_zoom2x_batched_noalloc(B.WENO_NOALLOC_MAX_IMAGES + 1, 1, 0, 1, 0, p, 0, 0, None)
    assert rc == B.WENO_ERANGE
