"""Seeded synthetic binary edge images -> int16 edge-point lists.

The paper's own test images (three natural 256x256 images after a Sobel
operator, Section 4.1) are not available, so every workload here is drawn from
a seed: straight segments rasterised with an integer DDA, plus salt-noise
pixels.  Points are de-duplicated and emitted in row-major order (y, then x),
so the line id of a point is its position in the list.

Determinism: every random number comes from a counter-based SplitMix64 stream
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), and every floating-point step uses only +, -, *, / and sqrt,
which IEEE 754 rounds correctly, so the same seed gives the same points on
x86_64 and aarch64.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
CONFIG_SEED_BASE = 0x5EED0000


def ceil_log2(v: int) -> int:
    """Smallest e >= 0 with 2**e >= v (v >= 1)."""
    v = int(v)
    if v < 1:
        raise ValueError("ceil_log2 needs v >= 1")
    return (v - 1).bit_length()


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """SplitMix64 stream: draw k is mix(seed + (k + 1) * golden)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)
        self.k = 0

    def u64(self, count: int) -> np.ndarray:
        idx = np.arange(self.k + 1, self.k + 1 + count, dtype=np.uint64)
        self.k += count
        with np.errstate(over="ignore"):
            return _mix(self.seed + idx * GOLDEN)

    def child(self, tag: int) -> "Stream":
        with np.errstate(over="ignore"):
            s = _mix(np.array([self.seed ^ (np.uint64(tag) * _M2)], dtype=np.uint64))[0]
        return Stream(int(s))

    def ints(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (multiply-shift; span < 2**32)."""
        span = np.uint64(hi - lo + 1)
        u = self.u64(count) >> np.uint64(32)
        return (np.int64(lo) + ((u * span) >> np.uint64(32)).astype(np.int64))

    def floats(self, count: int) -> np.ndarray:
        """Uniform doubles in [0, 1) with 53 random bits."""
        return (self.u64(count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass
class EdgeImage:
    name: str
    W: int
    H: int
    depth: int
    T: int
    points: np.ndarray  # int16 [n, 2], columns (x, y)
    seed: int
    noise: float = 0.0
    segments: int = 0

    @property
    def n(self) -> int:
        return int(self.points.shape[0])


def _raster(segs: np.ndarray, W: int, H: int) -> np.ndarray:
    """Integer DDA rasterisation of segments [k, 4] = (x0, y0, x1, y1).

    Step t of N = max(|dx|, |dy|) lands on x0 + sgn(dx) * floor((2 t |dx| + N) / 2N)
    (the Bresenham pixel set up to tie-breaking).  Pixels outside the image are
    dropped.  Returns linear pixel indices y * W + x.
    """
    if segs.size == 0:
        return np.zeros(0, dtype=np.int64)
    x0, y0, x1, y1 = (segs[:, c].astype(np.int64) for c in range(4))
    dx, dy = x1 - x0, y1 - y0
    N = np.maximum(np.abs(dx), np.abs(dy))
    reps = N + 1
    seg_id = np.repeat(np.arange(len(N)), reps)
    starts = np.cumsum(reps) - reps
    t = np.arange(int(reps.sum()), dtype=np.int64) - np.repeat(starts, reps)
    Ns = np.maximum(N[seg_id], 1)
    ax, ay = np.abs(dx)[seg_id], np.abs(dy)[seg_id]
    px = x0[seg_id] + np.sign(dx)[seg_id] * ((2 * t * ax + Ns) // (2 * Ns))
    py = y0[seg_id] + np.sign(dy)[seg_id] * ((2 * t * ay + Ns) // (2 * Ns))
    keep = (px >= 0) & (px < W) & (py >= 0) & (py < H)
    return py[keep] * W + px[keep]


def _unit_dirs(st: Stream, count: int) -> np.ndarray:
    """Uniform directions by rejection in the unit disc (no trig functions)."""
    out = np.zeros((count, 2), dtype=np.float64)
    filled = 0
    while filled < count:
        want = 2 * (count - filled) + 8
        uv = st.floats(2 * want).reshape(want, 2) * 2.0 - 1.0
        r2 = uv[:, 0] * uv[:, 0] + uv[:, 1] * uv[:, 1]
        ok = uv[(r2 > 1e-12) & (r2 <= 1.0)]
        ok = ok / np.sqrt(ok[:, 0] * ok[:, 0] + ok[:, 1] * ok[:, 1])[:, None]
        take = min(count - filled, len(ok))
        out[filled:filled + take] = ok[:take]
        filled += take
    return out


def edge_points(W: int, H: int, segs: np.ndarray, noise: float, st: Stream) -> np.ndarray:
    """Union of rasterised segments and round(noise * W * H) uniform noise
    pixels (drawn with replacement), as row-major int16 (x, y) points."""
    pix = [_raster(segs, W, H)]
    m_exact = noise * W * H
    m = int(np.floor(m_exact + st.floats(1)[0]))
    if m > 0:
        pix.append(st.ints(0, W * H - 1, m))
    # the distinct pixel indices in increasing order (a mask of the image:
    # the same result as np.unique, without its hashing)
    mask = np.zeros(W * H, dtype=bool)
    for part in pix:
        mask[part] = True
    lin = np.flatnonzero(mask)
    pts = np.empty((lin.size, 2), dtype=np.int16)
    pts[:, 0] = (lin % W).astype(np.int16)
    pts[:, 1] = (lin // W).astype(np.int16)
    return pts


def _segments_uniform_endpoints(st: Stream, k: int, W: int, H: int) -> np.ndarray:
    xs = st.ints(0, W - 1, 2 * k).reshape(k, 2)
    ys = st.ints(0, H - 1, 2 * k).reshape(k, 2)
    return np.stack([xs[:, 0], ys[:, 0], xs[:, 1], ys[:, 1]], axis=1)


def _segments_by_length(st: Stream, k: int, W: int, H: int, lmin: int, lmax: int) -> np.ndarray:
    x0 = st.ints(0, W - 1, k)
    y0 = st.ints(0, H - 1, k)
    ln = st.ints(lmin, lmax, k).astype(np.float64)
    d = _unit_dirs(st, k)
    x1 = x0 + np.floor(ln * d[:, 0] + 0.5).astype(np.int64)
    y1 = y0 + np.floor(ln * d[:, 1] + 0.5).astype(np.int64)
    return np.stack([x0, y0, x1, y1], axis=1)


def _log_uniform_side(st: Stream, lo: int, hi: int, count: int) -> np.ndarray:
    """Integer sides with P(s) proportional to 1/s on [lo, hi] (discrete log-uniform)."""
    sides = np.arange(lo, hi + 1, dtype=np.int64)
    w = 1.0 / sides.astype(np.float64)
    cdf = np.cumsum(w)
    u = st.floats(count) * cdf[-1]
    return sides[np.minimum(np.searchsorted(cdf, u, side="right"), len(sides) - 1)]


def plain_128(index: int = 0, seed: Optional[int] = None) -> EdgeImage:
    """128x128, 4 segments with uniform endpoints, 1% salt noise; depth 7, T = 20."""
    seed = CONFIG_SEED_BASE + 0 if seed is None else seed
    st = Stream(seed).child(index)
    segs = _segments_uniform_endpoints(st, 4, 128, 128)
    pts = edge_points(128, 128, segs, 0.01, st)
    return EdgeImage("plain_128", 128, 128, 7, 20, pts, seed, 0.01, 4)


def plain_1024(index: int = 0, seed: Optional[int] = None) -> EdgeImage:
    """1024x1024, 32 segments of length 100-1000 px, 2% salt noise; depth 10, T = 64."""
    seed = CONFIG_SEED_BASE + 1 if seed is None else seed
    st = Stream(seed).child(index)
    segs = _segments_by_length(st, 32, 1024, 1024, 100, 1000)
    pts = edge_points(1024, 1024, segs, 0.02, st)
    return EdgeImage("plain_1024", 1024, 1024, 10, 64, pts, seed, 0.02, 32)


def plain_4096(index: int = 0, seed: Optional[int] = None) -> EdgeImage:
    """4096x4096, 512 segments of length 50-4000 px, 1% salt noise; depth 12, T = 128."""
    seed = CONFIG_SEED_BASE + 3 if seed is None else seed
    st = Stream(seed).child(index)
    segs = _segments_by_length(st, 512, 4096, 4096, 50, 4000)
    pts = edge_points(4096, 4096, segs, 0.01, st)
    return EdgeImage("plain_4096", 4096, 4096, 12, 128, pts, seed, 0.01, 512)


def batch_image(k: int, seed: Optional[int] = None) -> EdgeImage:
    """Image k of the mixed batch: side log-uniform in 256-2048 (square),
    8-64 segments with uniform endpoints, noise uniform in 0.5-5%,
    depth ceil(log2 side), T = floor(2 * side / 32)."""
    seed = CONFIG_SEED_BASE + 2 if seed is None else seed
    st = Stream(seed).child(k)
    s = int(_log_uniform_side(st, 256, 2048, 1)[0])
    nseg = int(st.ints(8, 64, 1)[0])
    p = 0.005 + 0.045 * float(st.floats(1)[0])
    segs = _segments_uniform_endpoints(st, nseg, s, s)
    pts = edge_points(s, s, segs, p, st)
    return EdgeImage(f"batch_256[{k}]", s, s, ceil_log2(s), max(1, (2 * s) // 32), pts, seed, p, nseg)


def batch_256(count: int = 256, seed: Optional[int] = None, first: int = 0) -> List[EdgeImage]:
    return [batch_image(first + k, seed) for k in range(count)]


def serving_request(k: int, seed: Optional[int] = None) -> EdgeImage:
    """Request k of the serving stream: side log-uniform in 64-4096, 1-256
    segments, noise uniform in 0-3%, depth ceil(log2 side), T uniform in 16-256."""
    seed = CONFIG_SEED_BASE + 4 if seed is None else seed
    st = Stream(seed).child(k)
    s = int(_log_uniform_side(st, 64, 4096, 1)[0])
    nseg = int(st.ints(1, 256, 1)[0])
    p = 0.03 * float(st.floats(1)[0])
    T = int(st.ints(16, 256, 1)[0])
    segs = _segments_uniform_endpoints(st, nseg, s, s)
    pts = edge_points(s, s, segs, p, st)
    return EdgeImage(f"serve[{k}]", s, s, ceil_log2(s), T, pts, seed, p, nseg)


def serving_requests(count: int, seed: Optional[int] = None, first: int = 0) -> List[EdgeImage]:
    return [serving_request(first + k, seed) for k in range(count)]


def poisson_arrivals(count: int, rate_per_s: float, seed: int = CONFIG_SEED_BASE + 5) -> np.ndarray:
    """Open-loop arrival times (s) of a Poisson process; only timing depends on these."""
    u = Stream(seed).floats(count)
    gaps = -np.log1p(-u) / float(rate_per_s)
    return np.cumsum(gaps)


def random_small(seed: int, max_side: int = 16, max_n: int = 64, max_depth: int = 5,
                 max_T: int = 8) -> EdgeImage:
    """Tiny random case for brute-force checks: W, H in [1, max_side], n points
    drawn uniformly (duplicates kept), depth in [1, max_depth], T in [1, max_T]."""
    st = Stream(seed)
    W = int(st.ints(1, max_side, 1)[0])
    H = int(st.ints(1, max_side, 1)[0])
    n = int(st.ints(0, max_n, 1)[0])
    D = int(st.ints(1, max_depth, 1)[0])
    T = int(st.ints(1, max_T, 1)[0])
    pts = np.stack([st.ints(0, W - 1, n), st.ints(0, H - 1, n)], axis=1).astype(np.int16)
    return EdgeImage(f"small[{seed}]", W, H, D, T, pts.reshape(n, 2), seed)
