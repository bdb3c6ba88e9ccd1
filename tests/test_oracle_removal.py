"""Pins of the oracle's solution() mode (Section 3: voters of an accepted leaf
are plotted and removed from every region reached later).

- a restatement from the definition on tiny inputs: regions visited depth
  first (NE, NW, SW, SE) by recursion, a set of points not yet plotted, and
  crossing decided on exact rational corners (the pins' Fraction vertex
  table, not the oracle's arithmetic); its accepted cells, statistics and
  plotted points must equal the oracle's;
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


def _crosses(below, i0, j0, S):
    """The line of a point crosses the region with corners (i0, j0) and
    (i0 + S, j0 + S): its corner code is neither 0000 nor 1111."""
    code = ((below[i0 + S][j0 + S] << 3) | (below[i0][j0 + S] << 2) | (below[i0][j0] << 1)
            | below[i0 + S][j0])
    return code not in (0, 15)


def _removal_by_definition(points, W, H, D, T):
    """solution() from its description: a plotted point takes no part in any
    region reached after its leaf.  Crossing is monotone (a line that crosses
    a region crosses every region containing it), so when a child is reached
    the points tested for it are the unplotted points that cross its parent,
    and its votes are those among them that cross the child.  A leaf that
    reaches T plots its voters at once.  Returns (leaves in visiting order,
    stats [2, D + 1, 4], plotted [2, n])."""
    L = pins.frame_side(W, H)
    K = 1 << D
    n = len(points)
    leaves = []
    plotted = np.zeros((2, n), np.uint8)
    stats = np.zeros((2, D + 1, 4), np.uint64)
    for half in (0, 1):
        pts = pins.half_points(points, half)
        below = [pins._vertex_below_table(int(x), int(y), L, K) for x, y in pts]
        live = np.ones(n, bool)
        root_votes = sum(1 for e in range(n) if _crosses(below[e], 0, 0, K))
        stats[half, 0] = (1, 1, root_votes, n)

        def visit(level, i0, j0, S):
            h = S // 2
            for ci, cj in ((i0 + h, j0 + h), (i0, j0 + h), (i0, j0), (i0 + h, j0)):
                tested = [e for e in range(n) if live[e] and _crosses(below[e], i0, j0, S)]
                voters = [e for e in tested if _crosses(below[e], ci, cj, h)]
                row = stats[half, level + 1]
                row[0] += 1
                row[2] += len(voters)
                row[3] += len(tested)
                if len(voters) < T:
                    continue
                row[1] += 1
                if level + 1 == D:
                    leaves.append((half, ci, cj, len(voters)))
                    live[voters] = False
                    plotted[half, voters] = 1
                else:
                    visit(level + 1, ci, cj, h)

        visit(0, 0, 0, K)
    return np.array(leaves, dtype=np.uint32).reshape(-1, 4), stats, plotted


@pytest.mark.parametrize("seed", range(40))
def test_against_the_definition_restated(seed):
    img = synth.random_small(81000 + seed, max_side=16, max_n=40, max_depth=4, max_T=4)
    want_leaves, want_stats, want_plotted = _removal_by_definition(img.points, img.W, img.H, img.depth, img.T)
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
