"""api.HostPipeline: frames from pinned host memory through the zoom and back,
with neighbouring frames' copies overlapped with the zoom.  Every output must
equal the plain per-frame call bit for bit."""
import pytest
import torch

from paper_2312_00229_gb300 import api, scenes

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,depth", [(torch.uint8, 3), (torch.float32, 2), (torch.uint8, 1)])
def test_pipeline_matches_plain_calls(dtype, depth):
    frames = []
    for i in range(7):
        img = scenes.planar(scenes.piecewise_smooth(90, 160, seed=scenes.seed_for(7, i),
                                                    scale_features=True))
        x = torch.from_numpy(img)
        frames.append((x if dtype == torch.uint8 else x.float() / 255.0).pin_memory())
    pipe = api.HostPipeline(tuple(frames[0].shape), dtype, device="cuda", depth=depth)
    outs = [torch.empty(pipe.out_shape, dtype=dtype).pin_memory() for _ in frames]
    for x, y in zip(frames, outs):
        pipe.submit(x, y)
    pipe.flush()
    for x, y in zip(frames, outs):
        ref = api.zoom2x_fwd(x.cuda()).cpu()
        assert torch.equal(y, ref)
