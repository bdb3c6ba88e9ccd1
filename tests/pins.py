"""Independent checks that pin the CPU oracle (no code shared with it).

brute_force():   the paper's definition taken literally.  Corner points are
                 exact rationals (fractions.Fraction) on the dyadic m/b grid;
                 each corner is classified with F = y0 - m*x0 - b of Section 2
                 (line slope m = -x, intercept b = y in parameter space); the
                 4-bit code is formed per cell in NE, NW, SW, SE order and every
                 cell of every level is counted directly over all points.  The
                 hierarchy rules (root always split, children of passed regions
                 tested, pass iff votes >= T) are then applied to those direct
                 counts.  No voter lists, no recursion.

column_counts(): a closed form.  For x >= 0 the scaled sign function is
                 non-decreasing in m and increasing in b, so a line votes for a
                 cell exactly when the SW corner is below it and the NE corner
                 is not; per column of cells that is an integer interval of b
                 indices, accumulated with a difference array.  O(n * 2^l) per
                 level, so it also runs on full-size images.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

import numpy as np


def frame_side(W: int, H: int) -> int:
    L = 1
    while L < max(W, H):
        L *= 2
    return L


def half_points(points: np.ndarray, half: int) -> np.ndarray:
    p = np.asarray(points, dtype=np.int64).reshape(-1, 2)
    return p if half == 0 else p[:, ::-1]


# --------------------------------------------------------------------------- brute force
def _vertex_below_table(x: int, y: int, L: int, K: int):
    """below[i][j] = True when grid vertex (m_i, b_j) lies strictly below the
    parameter-space line of edge point (x, y)."""
    ms = [Fraction(-1) + Fraction(2 * i, K) for i in range(K + 1)]
    bs = [Fraction(-2 * L) + Fraction(4 * L * j, K) for j in range(K + 1)]
    slope, intercept = -x, y  # b = y - x*m  <=>  "y = m x + b" with m := -x, b := y
    out = []
    for m0 in ms:
        row = []
        for b0 in bs:
            F = b0 - slope * m0 - intercept  # F(x0, y0) = y0 - m*x0 - b with (x0, y0) = (m0, b0)
            row.append(F < 0)
        out.append(row)
    return out


def brute_force(points, W: int, H: int, D: int, T: int):
    """Returns (leaves as sorted list of (half, i, j, votes), stats[2][D+1][4])."""
    L = frame_side(W, H)
    K = 2 ** D
    stats = np.zeros((2, D + 1, 4), dtype=np.int64)
    leaves = []
    table = lru_cache(maxsize=None)(lambda x, y: _vertex_below_table(x, y, L, K))
    for half in (0, 1):
        pts = [tuple(map(int, p)) for p in half_points(points, half)]
        passed_prev = None
        for level in range(D + 1):
            S = K >> level
            cells = 1 << level
            counts = np.zeros((cells, cells), dtype=np.int64)
            for (x, y) in pts:
                below = table(x, y)
                for a in range(cells):
                    for b in range(cells):
                        i0, j0 = a * S, b * S
                        code = ((below[i0 + S][j0 + S] << 3) | (below[i0][j0 + S] << 2)
                                | (below[i0][j0] << 1) | below[i0 + S][j0])
                        if code != 0 and code != 15:
                            counts[a, b] += 1
            if level == 0:
                tested = np.ones((1, 1), dtype=bool)
                passed = np.ones((1, 1), dtype=bool)  # the root is always split
                stats[half, 0] = (1, 1, counts[0, 0], len(pts))
            else:
                tested = np.kron(passed_prev, np.ones((2, 2), dtype=bool))
                passed = tested & (counts >= T)
                parent_counts = prev_counts[passed_prev].sum()
                stats[half, level] = (tested.sum(), passed.sum(), counts[tested].sum(), 4 * parent_counts)
            if level == D:
                for a, b in zip(*np.nonzero(passed)):
                    leaves.append((half, int(a), int(b), int(counts[a, b])))
            passed_prev, prev_counts = passed, counts
    leaves.sort()
    return leaves, stats


# --------------------------------------------------------------------------- closed form
def _ceil_div(p: np.ndarray, q: int) -> np.ndarray:
    return -((-p) // q)


def column_counts(points, W: int, H: int, D: int, level: int, half: int) -> np.ndarray:
    """Direct vote count of every cell of `level` (shape [2^l, 2^l], index [a, b])
    from the per-column b-interval of each line."""
    L = frame_side(W, H)
    K = 2 ** D
    S = K >> level
    cells = 1 << level
    p = half_points(points, half)
    counts = np.zeros((cells, cells + 1), dtype=np.int64)
    if p.shape[0] == 0:
        return counts[:, :cells]
    x = p[:, 0][:, None]
    y = p[:, 1][:, None]
    chunk = max(1, (1 << 22) // max(1, p.shape[0]))
    for a0 in range(0, cells, chunk):
        a = np.arange(a0, min(cells, a0 + chunk), dtype=np.int64)[None, :]
        # SW corner (aS, bS) strictly below:  4L*b*S < 2LK + K(x+y) - 2x*a*S
        num_lo = 2 * L * K + K * (x + y) - 2 * x * a * S
        b_hi = _ceil_div(num_lo, 4 * L * S) - 1
        # NE corner ((a+1)S, (b+1)S) not below: 4L(b+1)S >= 2LK + K(x+y) - 2x(a+1)S
        num_ne = 2 * L * K + K * (x + y) - 2 * x * (a + 1) * S
        b_lo = _ceil_div(num_ne, 4 * L * S) - 1
        b_lo = np.clip(b_lo, 0, cells)
        b_hi = np.clip(b_hi, -1, cells - 1)
        ok = b_hi >= b_lo
        cols = np.broadcast_to(a, ok.shape)[ok]
        width = cells + 1
        flat = counts.reshape(-1)
        flat += np.bincount(cols * width + b_lo[ok], minlength=flat.size)
        flat -= np.bincount(cols * width + b_hi[ok] + 1, minlength=flat.size)
    return np.cumsum(counts, axis=1)[:, :cells]


def closed_form(points, W: int, H: int, D: int, T: int):
    """Hierarchy rules applied to column_counts() at every level."""
    n = int(np.asarray(points).reshape(-1, 2).shape[0])
    stats = np.zeros((2, D + 1, 4), dtype=np.int64)
    leaves = []
    for half in (0, 1):
        passed_prev = None
        prev_counts = None
        for level in range(D + 1):
            counts = column_counts(points, W, H, D, level, half)
            if level == 0:
                passed = np.ones((1, 1), dtype=bool)
                stats[half, 0] = (1, 1, counts[0, 0], n)
            else:
                tested = np.kron(passed_prev, np.ones((2, 2), dtype=bool))
                passed = tested & (counts >= T)
                stats[half, level] = (tested.sum(), passed.sum(), counts[tested].sum(),
                                      4 * prev_counts[passed_prev].sum())
            if level == D:
                for a, b in zip(*np.nonzero(passed)):
                    leaves.append((half, int(a), int(b), int(counts[a, b])))
            passed_prev, prev_counts = passed, counts
    leaves.sort()
    return leaves, stats


def dfs_key(i: int, j: int, depth: int) -> int:
    """Position of leaf cell (i, j) in the depth-first order of Section 3:
    at each level the child digit is quad1..quad4 = NE, NW, SW, SE."""
    key = 0
    for l in range(depth - 1, -1, -1):
        east, north = (i >> l) & 1, (j >> l) & 1
        q = (0 if east else 1) if north else (3 if east else 2)
        key = key * 4 + q
    return key


def dfs_keys(leaves: np.ndarray, depth: int) -> np.ndarray:
    """Vectorised (half, dfs_key) as one int64 per leaf row (half, i, j, votes)."""
    lv = np.asarray(leaves, dtype=np.int64).reshape(-1, 4)
    key = np.zeros(len(lv), dtype=np.int64)
    for l in range(depth - 1, -1, -1):
        east, north = (lv[:, 1] >> l) & 1, (lv[:, 2] >> l) & 1
        q = np.where(north == 1, np.where(east == 1, 0, 1), np.where(east == 1, 3, 2))
        key = key * 4 + q
    return (lv[:, 0] << 50) | key
