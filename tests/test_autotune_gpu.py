"""The autotuner times every (band height, tile width) candidate, caches the
fastest per size class, and the cached shape changes no output bit: tiles of
any shape compute the same values."""
import pytest
import torch

from paper_2312_00229_gb300 import api, autotune

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture
def fresh_cache(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE_PATH", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune, "_cache", None)
    yield


def test_tune_fwd_caches_a_shape_that_keeps_the_output(fresh_cache):
    g = torch.Generator(device=DEV).manual_seed(21)
    x = torch.randint(0, 256, (3, 90, 300), device=DEV, generator=g, dtype=torch.uint8)
    want = api.zoom2x_fwd(x, rows_per_tile=0)
    times = autotune.tune_fwd(x, candidates=(0, 16, 64), reps=2)
    assert set(times) == {(r, w) for r in (0, 16, 64) for w in (0, 247, 119, 246, 118)}
    best = min(times, key=times.get)
    assert autotune.lookup(x, x.dtype, "chw") == best[0]
    assert autotune.lookup_width(x, x.dtype, "chw") == best[1]
    got = api.zoom2x_fwd(x)  # the cached shape
    torch.cuda.synchronize()
    assert torch.equal(got, want)


def test_tune_batched_caches_a_shape_that_keeps_the_outputs(fresh_cache):
    g = torch.Generator(device=DEV).manual_seed(22)
    imgs = [torch.rand(3, h, w, device=DEV, generator=g).half()
            for h, w in [(40, 70), (130, 260), (9, 500)]]
    want = api.zoom2x_batched(imgs, rows_per_tile=0)
    times = autotune.tune_batched(imgs, candidates=(16, 64), reps=2)
    assert set(times) == {(r, w) for r in (16, 64) for w in (247, 119, 246, 118)}
    assert autotune.lookup_batched(imgs, None, "chw") == min(times, key=times.get)
    got = api.zoom2x_batched(imgs)  # the cached shape
    torch.cuda.synchronize()
    for a, b in zip(got, want):
        assert torch.equal(a, b)


def test_tune_cascade_keeps_every_output_bit(fresh_cache):
    """Tuning each level of a cascade caches a shape per level's size class;
    the cascade then runs with them and gives the same bits."""
    g = torch.Generator(device=DEV).manual_seed(22)
    x = torch.randint(0, 256, (3, 70, 90), device=DEV, generator=g, dtype=torch.uint8)
    want = api.cascade_zoom(x, 3)  # library default shapes (empty cache)
    times = autotune.tune_cascade(x, 3, candidates=(0, 16, 64), reps=2)
    assert len(times) == 3 and all(len(t) == 3 * 5 for t in times)
    got = api.cascade_zoom(x, 3)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    # with every level cached, only_missing times nothing and keeps the shapes
    before = dict(autotune._load())
    again = autotune.tune_cascade(x, 3, candidates=(0, 16), reps=1, only_missing=True)
    assert again == [{}, {}, {}] and autotune._load() == before
