"""Pins of the oracle's solution() mode (Section 3: voters of an accepted leaf
are plotted and removed from every region reached later).

- the paper's pseudocode written out literally on tiny inputs: per-level
  linecode arrays over all edge points, level.quad / level.vote, and
  solution() zeroing a plotted point's codes at every level; its accepted
  cells, statistics and plotted points must equal the oracle's;
- a hand-worked case: eight collinear points whose lines meet at a grid
  vertex fill two cells with 8 votes each; the first in depth-first order
  (NE before NW) takes all eight points and the second is left with none;
- invariants: accepted cells are order-free leaves with no more votes; the
  votes of a half's accepted cells add up to its plotted points; T > n
  plots nothing.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pins


def _pseudocode(points, W, H, D, T):
    """Section 3's algorithm as printed, one half after the other."""
    L = oracle.frame_side(W, H)
    K = 1 << D
    leaves, plotted = [], np.zeros((2, len(points)), np.uint8)
    stats = np.zeros((2, D + 1, 4), np.uint64)
    for half in (0, 1):
        pts = pins.half_points(points, half)
        E = len(pts)
        code = np.zeros((D + 1, E), np.int64)
        for e in range(E):
            code[0, e] = oracle.getcode(int(pts[e, 0]), int(pts[e, 1]), 0, 0, K, L, D)
        stats[half, 0] = (1, 1, sum(1 for e in range(E) if code[0, e] not in (0, 15)), E)
        region = {0: (0, 0, K)}
        quad = {1: 0}
        level = 1
        while level > 0:
            quad[level] += 1
            if quad[level] <= 4:
                i0, j0, S = region[level - 1]
                h = S // 2
                q = quad[level] - 1  # quad1..quad4 = NE, NW, SW, SE
                ci = i0 + (h if q in (0, 3) else 0)
                cj = j0 + (h if q in (0, 1) else 0)
                vote = 0
                evaluated = 0
                for e in range(E):
                    if code[level - 1, e] not in (0, 15):
                        evaluated += 1
                        c = oracle.getcode(int(pts[e, 0]), int(pts[e, 1]), ci, cj, h, L, D)
                        code[level, e] = c
                        if c not in (0, 15):
                            vote += 1
                    else:
                        code[level, e] = 0
                stats[half, level, 0] += 1
                stats[half, level, 2] += vote
                stats[half, level, 3] += evaluated
                if vote >= T:
                    stats[half, level, 1] += 1
                    if level == D:
                        leaves.append((half, ci, cj, vote))
                        for e in range(E):  # solution(): plot and zero the codes at every level
                            if code[D, e] not in (0, 15):
                                plotted[half, e] = 1
                                code[:, e] = 0
                    else:
                        region[level] = (ci, cj, h)
                        level += 1
                        quad[level] = 0
            else:
                level -= 1
    return np.array(leaves, dtype=np.uint32).reshape(-1, 4), stats, plotted


@pytest.mark.parametrize("seed", range(40))
def test_against_the_pseudocode_written_out(seed):
    img = synth.random_small(81000 + seed, max_side=16, max_n=40, max_depth=4, max_T=4)
    want_leaves, want_stats, want_plotted = _pseudocode(img.points, img.W, img.H, img.depth, img.T)
    got, plotted = oracle.detect_removal(img.points, img.W, img.H, img.depth, img.T)
    assert np.array_equal(got.leaves, want_leaves), seed
    assert np.array_equal(got.stats, want_stats), seed
    assert np.array_equal(plotted, want_plotted), seed


def test_hand_worked_concurrent_lines():
    pts = np.array([[x, 4] for x in range(8)], dtype=np.int16)
    # order-free: the cells with NE and NW corners at the vertex (4, 5) both get 8
    free = oracle.detect(pts, 8, 8, 3, 8)
    h0 = [tuple(int(v) for v in r) for r in free.leaves if r[0] == 0]
    assert (0, 3, 4, 8) in h0 and (0, 4, 4, 8) in h0
    got, plotted = oracle.detect_removal(pts, 8, 8, 3, 8)
    g0 = [tuple(int(v) for v in r) for r in got.leaves if r[0] == 0]
    assert g0 == [(0, 4, 4, 8)]          # NE of the top-level split is reached first
    assert plotted[0].sum() == 8          # all eight points plotted there


@pytest.mark.parametrize("k", range(3))
def test_invariants(k):
    img = synth.plain_128(index=k)
    got, plotted = oracle.detect_removal(img.points, img.W, img.H, img.depth, img.T)
    free = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    fmap = {(int(h), int(i), int(j)): int(v) for h, i, j, v in free.leaves}
    for h, i, j, v in got.leaves:
        assert fmap[(int(h), int(i), int(j))] >= int(v) >= img.T
    for half in (0, 1):
        assert int(got.leaves[got.leaves[:, 0] == half, 3].sum()) == int(plotted[half].sum())
    none, p0 = oracle.detect_removal(img.points, img.W, img.H, img.depth, img.n + 1)
    assert len(none.leaves) == 0 and p0.sum() == 0
