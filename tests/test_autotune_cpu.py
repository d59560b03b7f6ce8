"""Host logic of the autotuner cache (no GPU): size classes round the sides
up to powers of two, misses return the library defaults (0), and cached
shapes survive a reload from the JSON file."""
import json

import pytest
import torch

from paper_2312_00229_gb300 import autotune


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "autotune.json"
    monkeypatch.setattr(autotune, "CACHE_PATH", str(path))
    monkeypatch.setattr(autotune, "_cache", None)
    monkeypatch.setattr(autotune, "_device_name", lambda device: "TestGPU")
    return path


def test_pow2():
    assert [autotune._pow2(v) for v in (1, 2, 3, 5, 64, 65, 1080, 1920)] == \
        [1, 2, 4, 8, 64, 128, 2048, 2048]


def test_size_class_rounds_sides(cache):
    a = torch.zeros(3, 1080, 1920, dtype=torch.uint8)
    b = torch.zeros(3, 1100, 2000, dtype=torch.uint8)
    c = torch.zeros(3, 1080, 2100, dtype=torch.uint8)
    ka = autotune.size_class(a, torch.uint8, "chw")
    assert ka == autotune.size_class(b, torch.uint8, "chw")
    assert ka != autotune.size_class(c, torch.uint8, "chw")
    assert ka != autotune.size_class(a, torch.float16, "chw")
    assert "TestGPU" in ka


def test_misses_return_library_defaults(cache):
    x = torch.zeros(3, 64, 64, dtype=torch.uint8)
    assert autotune.lookup(x, torch.uint8, "chw") == 0
    assert autotune.lookup_width(x, torch.uint8, "chw") == 0
    assert autotune.lookup_batched([x, x], None, "chw") == (0, 0)


def test_cached_shapes_survive_a_reload(cache, monkeypatch):
    x = torch.zeros(3, 100, 500, dtype=torch.uint8)
    imgs = [x] * 5
    key = autotune.size_class(x, torch.uint8, "chw")
    bkey = autotune._batched_key(imgs, None, "chw")
    store = autotune._load()
    store[key], store[key + "|tile_width"] = 48, 119
    store[bkey], store[bkey + "|tile_width"] = 96, 247
    autotune._save()
    on_disk = json.loads(cache.read_text())
    assert on_disk[key] == 48 and on_disk[bkey + "|tile_width"] == 247
    monkeypatch.setattr(autotune, "_cache", None)  # force a reload from the file
    assert autotune.lookup(x, torch.uint8, "chw") == 48
    assert autotune.lookup_width(x, torch.uint8, "chw") == 119
    assert autotune.lookup_batched(imgs, None, "chw") == (96, 247)
    # the batched key depends on the image count's power of two: 5 -> 8
    assert autotune.lookup_batched([x] * 7, None, "chw") == (96, 247)
    assert autotune.lookup_batched([x] * 9, None, "chw") == (0, 0)
