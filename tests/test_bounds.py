"""Pins of the hard upper bounds that size the graph form's buffers and the
serving engine's admission (Section 2's membership test): at level l the
line of an edge point votes in at most

    min(4^l, 2^l + floor((W_h - 1) * 2^l / (2L)) + 2)

cells, where W_h is the image's extent along the half's x (W for half 0, H
for half 1) and L the frame side; a half's passed regions at level l are then
at most min(4^l, n * that / T).

The crossed cells are counted by brute force over every cell of the level,
on exact integer corner values (a cell is crossed when its corner code is
neither 0000 nor 1111), so the bound's derivation (a column's crossed cells
form one interval, and the intervals telescope) is checked rather than
restated; the oracle's per-level statistics must respect the bounds too.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pins


def _bound(l, Wh, L):
    col = 1 << l
    return min(col + (Wh - 1) * col // (2 * L) + 2, col * col)


def _crossed_cells(x, y, l, L):
    """Cells of the 2^l x 2^l grid of level l that the line of (x, y) crosses.
    Corner values are K * F scaled to the level's grid (K = 2^l): a vertex
    (a, b) lies below the line when 4L b + 2x a - 2L 2^l - 2^l x - 2^l y < 0."""
    col = 1 << l
    a = np.arange(col + 1, dtype=np.int64)[:, None]
    b = np.arange(col + 1, dtype=np.int64)[None, :]
    below = (4 * L * b + 2 * x * a - 2 * L * col - col * x - col * y) < 0
    s = (below[:-1, :-1].astype(np.int8) + below[1:, :-1] + below[:-1, 1:] + below[1:, 1:])
    return int(((s > 0) & (s < 4)).sum())


@pytest.mark.parametrize("W,H", [(1, 1), (7, 300), (128, 128), (300, 7), (1000, 999), (2023, 2021), (4096, 4096)])
def test_a_line_crosses_no_more_cells_than_the_bound(W, H):
    rng = np.random.default_rng(W * 7919 + H)
    L = pins.frame_side(W, H)
    worst_gap = None
    for half, (Wh, Hh) in enumerate(((W, H), (H, W))):
        xs = [0, Wh - 1] + [int(v) for v in rng.integers(0, Wh, 6)]
        ys = [0, Hh - 1] + [int(v) for v in rng.integers(0, Hh, 6)]
        for x in xs:
            for y in ys:
                for l in range(0, 9):
                    got, bound = _crossed_cells(x, y, l, L), _bound(l, Wh, L)
                    assert got <= bound, (half, x, y, l, got, bound)
                    if l >= 4:
                        gap = bound - got
                        worst_gap = gap if worst_gap is None else min(worst_gap, gap)
    # the bound is close: some line comes within 2 cells of it at a deep level
    assert worst_gap is not None and worst_gap <= 2, worst_gap


@pytest.mark.parametrize("seed", range(12))
def test_the_oracle_statistics_respect_the_bounds(seed):
    img = synth.random_small(87000 + seed, max_side=200, max_n=400, max_depth=8, max_T=5) if seed < 10 \
        else synth.plain_128(index=seed - 10)
    res = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    L = pins.frame_side(img.W, img.H)
    n = len(img.points)
    for half, Wh in enumerate((img.W, img.H)):
        for l in range(img.depth + 1):
            tested, passed, votes, _ = (int(v) for v in res.stats[half, l])
            assert votes <= n * _bound(l, Wh, L), (half, l)
            assert passed <= min(4 ** l, n * _bound(l, Wh, L) // img.T), (half, l)
            assert tested <= 4 ** l
