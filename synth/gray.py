"""Seeded synthetic grey-level images for the front end (Sobel edges and the
ALPHA/BETA split).

The paper's test images (three natural 256x256 pictures, Section 4.1) are not
available.  These stand in for them: a noisy background, filled rectangles
(step edges in both directions) and straight line segments drawn bright on
it, so that Sobel's operator finds edge points of every orientation.  Nothing
here computes a gradient: the generator only draws pixels.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from .edges import CONFIG_SEED_BASE, Stream, _raster, _segments_by_length, _segments_uniform_endpoints, ceil_log2


@dataclasses.dataclass
class GrayImage:
    name: str
    W: int
    H: int
    pixels: np.ndarray  # uint8 [H, W], row-major
    threshold: int      # Sobel magnitude threshold
    depth: int
    T: int
    seed: int


def gray_image(W: int, H: int, n_rects: int, segs: np.ndarray, noise_amp: int, st: Stream) -> np.ndarray:
    """Background uniform in [0, noise_amp]; rectangles of one grey level in
    [100, 200] each; segments (1 pixel wide) at 255."""
    img = st.ints(0, noise_amp, W * H).astype(np.uint8).reshape(H, W)
    for _ in range(n_rects):
        x0, x1 = np.sort(st.ints(0, W - 1, 2))
        y0, y1 = np.sort(st.ints(0, H - 1, 2))
        level = int(st.ints(100, 200, 1)[0])
        img[y0:y1 + 1, x0:x1 + 1] = level
    lin = _raster(segs, W, H)
    img.reshape(-1)[lin] = 255
    return img


def gray_256(index: int = 0, seed: Optional[int] = None) -> GrayImage:
    """256x256 (the paper's image size): 6 rectangles, 12 segments with uniform
    endpoints, background noise 0-30; Sobel threshold 200, depth 8, T = 20."""
    seed = CONFIG_SEED_BASE + 6 if seed is None else seed
    st = Stream(seed).child(index)
    segs = _segments_uniform_endpoints(st, 12, 256, 256)
    img = gray_image(256, 256, 6, segs, 30, st)
    return GrayImage("gray_256", 256, 256, img, 200, 8, 20, seed)


def gray_4096(index: int = 0, seed: Optional[int] = None) -> GrayImage:
    """4096x4096: 64 rectangles, 256 segments of length 50-4000, background
    noise 0-30; Sobel threshold 200, depth 12, T = 128."""
    seed = CONFIG_SEED_BASE + 7 if seed is None else seed
    st = Stream(seed).child(index)
    segs = _segments_by_length(st, 256, 4096, 4096, 50, 4000)
    img = gray_image(4096, 4096, 64, segs, 30, st)
    return GrayImage("gray_4096", 4096, 4096, img, 200, 12, 128, seed)


def gray_random(seed: int, max_side: int = 64) -> GrayImage:
    """Small random case: W, H in [1, max_side], a few rectangles and segments,
    threshold in [0, 400], depth ceil(log2 max(W, H)) (at least 1), T in [1, 8]."""
    st = Stream(seed)
    W = int(st.ints(1, max_side, 1)[0])
    H = int(st.ints(1, max_side, 1)[0])
    segs = _segments_uniform_endpoints(st, int(st.ints(0, 6, 1)[0]), W, H)
    img = gray_image(W, H, int(st.ints(0, 4, 1)[0]), segs, int(st.ints(0, 60, 1)[0]), st)
    thr = int(st.ints(0, 400, 1)[0])
    T = int(st.ints(1, 8, 1)[0])
    return GrayImage(f"gray_random[{seed}]", W, H, img, thr, max(1, ceil_log2(max(W, H))), T, seed)
