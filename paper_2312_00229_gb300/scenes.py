"""Seeded synthetic inputs for the WD WENO 2x zoom.

This module draws test images only; it holds none of the method's arithmetic
and is shared by the CUDA path's tests/benchmark and by the oracle's tests.
Every generator takes an explicit seed and returns a NumPy array; nothing here
touches the GPU.

The paper's own image workloads (a natural-image suite, a rasterised vector
drawing and pixel-art images) are not available here; these generators give
inputs of the same kind and size instead:

* ``analytic_step``: ``sin(2 pi x) cos(3 pi y) + [y >= 0.3 x + 0.4]`` at pixel
  centres of an n x n grid on [0, 1]^2 (x along columns, y along rows).
* ``piecewise_smooth``: an RGB scene of Gaussian bumps, hard-edged filled
  polygons, one-pixel lines and sensor noise (uint8).
* ``pixel_art``: a 16-colour palette image of 8x8 blocks with jagged
  diagonal one-pixel lines (uint8).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 2312_00229


def seed_for(config_index: int, image_index: int = 0) -> int:
    return BASE_SEED + 1000 * int(config_index) + int(image_index)


def rng_for(config_index: int, image_index: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config_index, image_index)))


# ----------------------------------------------------------------------------
# Analytic smooth + step function
# ----------------------------------------------------------------------------
def analytic_step(n: int = 64, with_step: bool = True) -> np.ndarray:
    """float64 [n, n]; sample (i, j) at x = (j + 1/2)/n, y = (i + 1/2)/n."""
    c = (np.arange(n) + 0.5) / n
    y = c[:, None]
    x = c[None, :]
    f = np.sin(2 * np.pi * x) * np.cos(3 * np.pi * y)
    if with_step:
        f = f + (y >= 0.3 * x + 0.4).astype(np.float64)
    return f


def analytic_step_truth(rows: int, cols: int, n: int, with_step: bool = True) -> np.ndarray:
    """The same function at fine positions x = (q + 1) / (2 n), y = (p + 1) / (2 n).

    Fine index p of a 2x zoom of the pixel-centre grid sits at
    y0 + p h / 2 with y0 = h / 2, h = 1 / n."""
    y = ((np.arange(rows) + 1.0) / (2 * n))[:, None]
    x = ((np.arange(cols) + 1.0) / (2 * n))[None, :]
    f = np.sin(2 * np.pi * x) * np.cos(3 * np.pi * y)
    if with_step:
        f = f + (y >= 0.3 * x + 0.4).astype(np.float64)
    return f


# ----------------------------------------------------------------------------
# Raster helpers
# ----------------------------------------------------------------------------
def _bresenham(r0: int, c0: int, r1: int, c1: int):
    """Integer points of the segment (r0, c0)-(r1, c1)."""
    pts = []
    dr, dc = abs(r1 - r0), abs(c1 - c0)
    sr = 1 if r1 >= r0 else -1
    sc = 1 if c1 >= c0 else -1
    err = dc - dr
    r, c = r0, c0
    while True:
        pts.append((r, c))
        if r == r1 and c == c1:
            break
        e2 = 2 * err
        if e2 > -dr:
            err -= dr
            c += sc
        if e2 < dc:
            err += dc
            r += sr
    return np.array(pts, dtype=np.int64)


def _draw_line(img: np.ndarray, r0, c0, r1, c1, colour):
    pts = _bresenham(int(r0), int(c0), int(r1), int(c1))
    H, W = img.shape[:2]
    keep = (pts[:, 0] >= 0) & (pts[:, 0] < H) & (pts[:, 1] >= 0) & (pts[:, 1] < W)
    pts = pts[keep]
    img[pts[:, 0], pts[:, 1]] = colour


def _fill_polygon(img: np.ndarray, verts: np.ndarray, colour):
    """Even-odd fill of pixels whose centres lie inside the polygon."""
    H, W = img.shape[:2]
    r_lo = max(int(np.floor(verts[:, 0].min())), 0)
    r_hi = min(int(np.ceil(verts[:, 0].max())), H - 1)
    c_lo = max(int(np.floor(verts[:, 1].min())), 0)
    c_hi = min(int(np.ceil(verts[:, 1].max())), W - 1)
    if r_lo > r_hi or c_lo > c_hi:
        return
    rr = (np.arange(r_lo, r_hi + 1) + 0.5)[:, None]
    cc = (np.arange(c_lo, c_hi + 1) + 0.5)[None, :]
    inside = np.zeros((rr.shape[0], cc.shape[1]), dtype=bool)
    k = len(verts)
    for a in range(k):
        ra, ca = verts[a]
        rb, cb = verts[(a + 1) % k]
        if ra == rb:
            continue
        crosses = (rr >= min(ra, rb)) & (rr < max(ra, rb))
        c_at = ca + (rr - ra) * (cb - ca) / (rb - ra)
        inside ^= crosses & (cc < c_at)
    region = img[r_lo:r_hi + 1, c_lo:c_hi + 1]
    region[inside] = colour


# ----------------------------------------------------------------------------
# Piecewise-smooth RGB scene
# ----------------------------------------------------------------------------
def piecewise_smooth(height: int, width: int, seed: int, channels: int = 3,
                     n_bumps: int = 32, n_polys: int = 64, n_lines: int = 128,
                     noise_sigma: float = 2.0, scale_features: bool = False) -> np.ndarray:
    """uint8 [height, width, channels] scene.

    32 Gaussian bumps (sigma 20-200 px, per-channel amplitude in [-60, 60] DN
    around a mid-grey of 128), 64 hard-edged filled polygons (3-8 vertices in
    a random box of side 20-400 px, random colours), 128 one-pixel lines with
    random end points and colours, additive Gaussian noise of `noise_sigma`
    DN, clipped to [0, 255] and rounded.  With ``scale_features`` the feature
    counts and sizes scale with the image (relative to 1920 x 1080)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H, W, C = int(height), int(width), int(channels)
    area_ratio = (H * W) / (1920.0 * 1080.0)
    size_ratio = np.sqrt(area_ratio)
    if scale_features:
        n_bumps = max(1, int(round(n_bumps * area_ratio)))
        n_polys = max(1, int(round(n_polys * area_ratio)))
        n_lines = max(1, int(round(n_lines * area_ratio)))
    else:
        size_ratio = 1.0
    img = np.full((H, W, C), 128.0, dtype=np.float64)
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    for _ in range(n_bumps):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        sig = rng.uniform(20, 200) * size_ratio
        amp = rng.uniform(-60, 60, size=C)
        gy = np.exp(-0.5 * ((yy - cy) / sig) ** 2)
        gx = np.exp(-0.5 * ((xx - cx) / sig) ** 2)
        img += (gy * gx)[:, :, None] * amp[None, None, :]
    for _ in range(n_polys):
        side = rng.uniform(20, 400) * size_ratio
        r0, c0 = rng.uniform(-side / 2, H - side / 2), rng.uniform(-side / 2, W - side / 2)
        k = int(rng.integers(3, 9))
        verts = np.stack([r0 + rng.uniform(0, side, k), c0 + rng.uniform(0, side, k)], axis=1)
        colour = rng.uniform(0, 255, size=C)
        _fill_polygon(img, verts, colour)
    for _ in range(n_lines):
        r0, r1 = rng.integers(0, H, size=2)
        c0, c1 = rng.integers(0, W, size=2)
        colour = rng.uniform(0, 255, size=C)
        _draw_line(img, r0, c0, r1, c1, colour)
    img += rng.normal(0.0, noise_sigma, size=img.shape)
    return np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8)


# ----------------------------------------------------------------------------
# Pixel art
# ----------------------------------------------------------------------------
def pixel_art(height: int, width: int, seed: int, channels: int = 3,
              block: int = 8, n_lines: int | None = None) -> np.ndarray:
    """uint8 [height, width, channels]: a random 16-colour palette, one palette
    colour per 8x8 block, then jagged one-pixel lines at slopes +-1, +-1/2 and
    +-2 in palette colours."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H, W, C = int(height), int(width), int(channels)
    palette = rng.integers(0, 256, size=(16, C)).astype(np.uint8)
    bh, bw = -(-H // block), -(-W // block)
    idx = rng.integers(0, 16, size=(bh, bw))
    img = palette[idx].repeat(block, axis=0).repeat(block, axis=1)[:H, :W].copy()
    if n_lines is None:
        n_lines = max(4, (H + W) // 32)
    slopes = [(1, 1), (1, -1), (1, 2), (1, -2), (2, 1), (2, -1)]
    for _ in range(n_lines):
        dr, dc = slopes[int(rng.integers(0, len(slopes)))]
        length = int(rng.integers(8, max(9, min(H, W) // 2)))
        r0, c0 = int(rng.integers(0, H)), int(rng.integers(0, W))
        r1 = r0 + dr * length // max(abs(dr), abs(dc))
        c1 = c0 + dc * length // max(abs(dr), abs(dc))
        _draw_line(img, r0, c0, r1, c1, palette[int(rng.integers(0, 16))])
    return img


# ----------------------------------------------------------------------------
# Workload bundles
# ----------------------------------------------------------------------------
def planar(img_hwc: np.ndarray) -> np.ndarray:
    """[H, W, C] -> contiguous [C, H, W]."""
    return np.ascontiguousarray(np.transpose(img_hwc, (2, 0, 1)))


def uneven_batch(count: int = 256, lo: int = 64, hi: int = 1024, config_index: int = 3,
                 channels: int = 3):
    """`count` uint8 [H, W, C] images, sides i.i.d. uniform in {lo..hi}; even
    indices are piecewise-smooth scenes scaled to the image, odd indices pixel
    art."""
    sizes_rng = rng_for(config_index, 999_999)
    hs = sizes_rng.integers(lo, hi + 1, size=count)
    ws = sizes_rng.integers(lo, hi + 1, size=count)
    imgs = []
    for i in range(count):
        s = seed_for(config_index, i)
        if i % 2 == 0:
            imgs.append(piecewise_smooth(int(hs[i]), int(ws[i]), s, channels, scale_features=True))
        else:
            imgs.append(pixel_art(int(hs[i]), int(ws[i]), s, channels))
    return imgs


def uneven_sizes(count: int = 256, lo: int = 64, hi: int = 1024, config_index: int = 3):
    sizes_rng = rng_for(config_index, 999_999)
    hs = sizes_rng.integers(lo, hi + 1, size=count)
    ws = sizes_rng.integers(lo, hi + 1, size=count)
    return [(int(a), int(b)) for a, b in zip(hs, ws)]
