"""Autotuner for the tile shape of the forward and batched zoom.

The CUDA kernels take the band height (coarse rows per CTA) as a run-time
parameter, and the strip width (output columns per CTA) as one of the built
tile shapes, which also fix the coarse columns per thread (the threads that
share one quad column's work): 247 (256 threads, one column each), 119 (128
threads, one column), 246 (128 threads, two columns each) or 118 (64
threads, two columns).  The one-launch forward picks a shape from the image
width; the batched launch takes one of the one-column widths from the
caller.  This module times candidate shapes
on the current GPU with CUDA events and caches the fastest per size class in
a JSON file, keyed by device name, storage types, layout and size class
(planes and the image sides rounded up to powers of two).

``api.zoom2x_fwd(..., rows_per_tile=None)`` consults the cache; a miss uses the
library's own default (the band count that balances the last wave of CTAs).
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Iterable, Optional, Sequence, Tuple

import torch

CACHE_PATH = os.environ.get(
    "WDWENO_AUTOTUNE_CACHE",
    os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json"))
CANDIDATES = (0, 16, 24, 32, 48, 64, 96, 128, 192)
# output columns per CTA: one column per thread (256 and 128 threads) and
# two columns per thread (128 and 64 threads)
TILE_WIDTHS = (247, 119, 246, 118)
BATCHED_TILE_WIDTHS = TILE_WIDTHS  # the persistent kernel runs either tile

_lock = threading.Lock()
_cache: Optional[Dict[str, int]] = None
_dev_names: Dict[int, str] = {}


def _device_name(device) -> str:
    idx = device.index if device.index is not None else torch.cuda.current_device()
    if idx not in _dev_names:
        _dev_names[idx] = torch.cuda.get_device_name(idx)
    return _dev_names[idx]


def _pow2(v: int) -> int:
    p = 1
    while p < v:
        p <<= 1
    return p


def size_class(x: torch.Tensor, out_dtype, layout: str) -> str:
    from .api import _planes
    h, w, c, _, _, _ = _planes(x, layout)
    dev = _device_name(x.device)
    return "|".join([dev, str(x.dtype), str(out_dtype), layout, str(_pow2(int(c))),
                     str(_pow2(int(h))), str(_pow2(int(w)))])


def _load() -> Dict[str, int]:
    global _cache
    with _lock:
        if _cache is None:
            try:
                with open(CACHE_PATH) as fh:
                    _cache = {k: int(v) for k, v in json.load(fh).items()}
            except (OSError, ValueError):
                _cache = {}
        return _cache


def _save() -> None:
    with _lock:
        os.makedirs(os.path.dirname(CACHE_PATH), exist_ok=True)
        tmp = CACHE_PATH + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(_cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, CACHE_PATH)


def lookup(x: torch.Tensor, out_dtype, layout: str) -> int:
    """Cached band height for this size class, or 0 (library default)."""
    return _load().get(size_class(x, out_dtype, layout), 0)


def lookup_width(x: torch.Tensor, out_dtype, layout: str) -> int:
    """Cached tile width for this size class, or 0 (the library's choice)."""
    return _load().get(size_class(x, out_dtype, layout) + "|tile_width", 0)


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_fwd(x: torch.Tensor, params=None, out_dtype=None, layout: str = "chw",
             candidates: Iterable[int] = CANDIDATES, widths: Iterable[int] = (0,) + TILE_WIDTHS,
             reps: int = 10) -> Dict[Tuple[int, int], float]:
    """Times each candidate (band height, tile width) on `x` and caches the
    fastest (width 0 = the library's choice for the image width).
    Returns {(rows_per_tile, tile_width): milliseconds}."""
    from . import api
    params = params or api.Params()
    odt = out_dtype or x.dtype
    out = api._out_like(x, params, layout, odt)
    times = {}
    for tw in widths:
        for r in candidates:
            times[(int(r), int(tw))] = _time(
                lambda: api.zoom2x_fwd(x, params, layout=layout, rows_per_tile=r, out=out,
                                       tile_width=tw), reps)
    best = min(times, key=times.get)
    key = size_class(x, odt, layout)
    _load()[key] = best[0]
    _load()[key + "|tile_width"] = best[1]
    _save()
    return times




def tune_cascade(x: torch.Tensor, levels: int, params=None, out_dtype=None,
                 inter_dtype=torch.float32, layout: str = "chw",
                 candidates: Iterable[int] = CANDIDATES, reps: int = 10,
                 only_missing: bool = False) -> list:
    """Tunes the tile shape of every level of ``api.cascade_zoom(x, levels)``
    (each level is its own size class: its input shape and storage pair),
    running the chain on `x` to get each level's input.  Returns the
    per-level timing dicts of ``tune_fwd`` (an empty dict for a level that
    `only_missing` left with its cached shape)."""
    import dataclasses

    from . import api
    params = params or api.Params()
    bounds = api._level_bounds(x, params, levels)
    cur, out = x, []
    for lvl in range(levels):
        last = lvl == levels - 1
        p = dataclasses.replace(params, h=params.h / (1 << lvl), data_bound=bounds[lvl])
        odt = (out_dtype or x.dtype) if last else inter_dtype
        if only_missing and size_class(cur, odt, layout) in _load():
            out.append({})
        else:
            out.append(tune_fwd(cur, p, out_dtype=odt, layout=layout, candidates=candidates,
                                reps=reps))
        cur = api.zoom2x_fwd(cur, p, out_dtype=odt, layout=layout)
    return out


def _batched_key(images: Sequence[torch.Tensor], out_dtype, layout: str) -> str:
    return "|".join(["batched", _device_name(images[0].device),
                     str(images[0].dtype), str(out_dtype or images[0].dtype), layout,
                     str(_pow2(len(images)))])


def tune_batched(images: Sequence[torch.Tensor], params=None, out_dtype=None,
                 layout: str = "chw", candidates: Iterable[int] = (16, 32, 64, 128),
                 widths: Iterable[int] = BATCHED_TILE_WIDTHS,
                 reps: int = 5) -> Dict[Tuple[int, int], float]:
    """Times the persistent batched launch for each (band height, tile width)
    and caches the fastest under the batch's size class (dtype, layout, image
    count).  Returns {(rows_per_tile, tile_width): milliseconds}."""
    from . import api
    times = {}
    for tw in widths:
        for r in candidates:
            plan = api.BatchedPlan(images, params, out_dtype, layout, rows_per_tile=r,
                                   tile_width=tw)
            times[(int(r), int(tw))] = _time(plan.run, reps)
    best = min(times, key=times.get)
    key = _batched_key(images, out_dtype, layout)
    _load()[key] = best[0]
    _load()[key + "|tile_width"] = best[1]
    _save()
    return times


def lookup_batched(images: Sequence[torch.Tensor], out_dtype,
                   layout: str) -> Tuple[int, int]:
    """Cached (band height, tile width) of this batch's size class, or (0, 0)
    (the library defaults)."""
    key = _batched_key(images, out_dtype, layout)
    cache = _load()
    return cache.get(key, 0), cache.get(key + "|tile_width", 0)
