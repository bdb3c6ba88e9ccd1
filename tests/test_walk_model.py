"""A plain-Python model of the GPU's solution() walk (Section 3), checked
against the oracle's removal mode on the CPU.

The kernel does not follow the oracle's steps: it splits a region's voters
into its four children's lists once, when the region is entered, and takes
a child's votes from its list's length while no point has been plotted since
(a recount of the entries not removed otherwise); the split of a region two
levels above the leaves also counts its 16 grandchildren, and that of a
region three levels above them its 64 great-grandchildren, so that a child
one or two levels above the leaves is entered only when one of its leaves
can reach T, its statistics following from the counts otherwise.  Its four
warps fill a child's list in an order that varies from run to run, so the
kernel relies on a list being used only as a set.

This model takes the same steps in the same order, with every list shuffled
after it is built, and must give the oracle's accepted cells, statistics and
plotted points exactly: the walk's shortcuts and the order-free lists are
checked here, apart from the CUDA code that implements them.  Crossing uses
the definition (corner code neither 0000 nor 1111) on exact integer corner
values; counts are keyed by absolute cell corners, not by the kernel's bit
layouts.
"""
import random

import numpy as np
import pytest

import oracle
import synth
from tests import pins

NE, NW, SW, SE = 0, 1, 2, 3


def _corner(i0, j0, h, q):
    """SW corner of quadrant q (side h) of the region at (i0, j0) of side 2h."""
    return i0 + (h if q in (NE, SE) else 0), j0 + (h if q in (NE, NW) else 0)


def _walk_model(points, W, H, D, T, rng):
    """Returns (leaves in visiting order, stats [2, D + 1, 4], plotted [2, n])."""
    L = pins.frame_side(W, H)
    K = 1 << D
    n = len(points)
    leaves = []
    stats = np.zeros((2, D + 1, 4), np.uint64)
    plotted = np.zeros((2, n), np.uint8)

    def mode_of(level):
        return 1 if level == D - 2 else (2 if level == D - 3 else 0)

    for half in (0, 1):
        p = pins.half_points(points, half)
        X, Y = [int(v) for v in p[:, 0]], [int(v) for v in p[:, 1]]

        def below(v, i, j):
            # K * F at grid vertex (i, j), negative when the vertex lies below the line
            return 4 * L * j + 2 * X[v] * i - 2 * L * K - K * X[v] - K * Y[v] < 0

        def crosses(v, i, j, s):
            code = below(v, i + s, j + s) + below(v, i, j + s) + below(v, i, j) + below(v, i + s, j)
            return 0 < code < 4

        removed = np.zeros(n, bool)
        st = stats[half]
        lists = {}
        counts = {1: {}, 2: {}, 3: {}}  # grandchildren (mode 1), grandchildren and leaves (mode 2)

        def split(src, check, level, i0, j0, h, mode):
            """The split of the region at (i0, j0) of side 2h entered at `level`:
            its children's lists (shuffled) and lengths, the voters not removed."""
            alive = [v for v in src if not (check and removed[v])]
            lens = []
            for q in range(4):
                ci, cj = _corner(i0, j0, h, q)
                lst = [v for v in alive if crosses(v, ci, cj, h)]
                rng.shuffle(lst)
                lists[(level, q)] = lst
                lens.append(len(lst))
            if mode:
                g = h // 2
                counts[mode] = {(i0 + a * g, j0 + b * g): sum(crosses(v, i0 + a * g, j0 + b * g, g) for v in alive)
                                for a in range(4) for b in range(4)}
            if mode == 2:
                e = h // 4
                counts[3] = {(i0 + a * e, j0 + b * e): sum(crosses(v, i0 + a * e, j0 + b * e, e) for v in alive)
                             for a in range(8) for b in range(8)}
            return len(alive), lens

        _, lens = split(list(range(n)), False, 0, 0, 0, K // 2, mode_of(0))
        st[0] = (1, 1, n, n)
        stack = [None] * (D + 1)
        stack[0] = {"q": 0, "i0": 0, "j0": 0, "lens": lens, "m": n, "rem": 0}
        plotted_count = 0
        level = 0
        while True:
            fr = stack[level]
            q = fr["q"]
            if q == 4:
                if level == 0:
                    break
                level -= 1
                continue
            fr["q"] = q + 1
            h = (K >> level) // 2
            ci, cj = _corner(fr["i0"], fr["j0"], h, q)
            cl = level + 1
            src = lists[(level, q)]
            ln = fr["lens"][q]
            evaluated = fr["m"] - (plotted_count - fr["rem"])
            stale = plotted_count != fr["rem"]
            cnt, clens, accounted = ln, [0, 0, 0, 0], False
            if cl == D:
                if stale:
                    cnt = sum(1 for v in src if not removed[v])
            elif cl == D - 2 and not stale:
                # counted in the parent's split: the child's children (side h / 2)
                # and their leaves (side h / 4)
                kids = [_corner(ci, cj, h // 2, k) for k in range(4)]
                can_pass = any(counts[2][c] >= T and any(counts[3][_corner(*c, h // 4, m)] >= T for m in range(4))
                               for c in kids)
                if can_pass and ln >= T:
                    cnt, clens = split(src, False, cl, ci, cj, h // 2, 1)
                else:
                    accounted = True
                    if ln >= T:
                        cv = cp = 0
                        for c in kids:
                            ck = counts[2][c]
                            cv += ck
                            if ck < T:
                                continue
                            cp += 1
                            st[D] += np.array([4, 0, sum(counts[3][_corner(*c, h // 4, m)] for m in range(4)), 4 * ck],
                                              np.uint64)
                        st[D - 1] += np.array([4, cp, cv, 4 * ln], np.uint64)
            elif cl == D - 1 and not stale:
                clens = [counts[1][_corner(ci, cj, h // 2, k)] for k in range(4)]
                if max(clens) >= T and ln >= T:
                    _, clens = split(src, False, cl, ci, cj, h // 2, 0)
            else:
                cnt, clens = split(src, stale, cl, ci, cj, h // 2, mode_of(cl))
            st[cl] += np.array([1, 0, cnt, evaluated], np.uint64)
            if cnt < T:
                continue
            st[cl][1] += 1
            if cl == D:
                leaves.append((half, ci, cj, cnt))
                removed[src] = True
                plotted_count += cnt
            elif accounted:
                pass
            elif cl == D - 1 and max(clens) < T:
                st[D] += np.array([4, 0, sum(clens), 4 * cnt], np.uint64)
            else:
                stack[cl] = {"q": 0, "i0": ci, "j0": cj, "lens": clens, "m": cnt, "rem": plotted_count}
                level = cl
        plotted[half] = removed
    return np.array(leaves, dtype=np.uint32).reshape(-1, 4), stats, plotted


def _check(img, seed):
    got_leaves, got_stats, got_plotted = _walk_model(img.points, img.W, img.H, img.depth, img.T,
                                                     random.Random(seed))
    want, want_plotted = oracle.detect_removal(img.points, img.W, img.H, img.depth, img.T)
    assert np.array_equal(got_leaves, want.leaves), img.name
    assert np.array_equal(got_stats, want.stats), img.name
    assert np.array_equal(got_plotted, want_plotted), img.name


@pytest.mark.parametrize("seed", range(60))
def test_model_matches_the_oracle_on_small_images(seed):
    """Depths 1-6 (so every shortcut level, including D <= 3 where the root's
    own split counts the leaves), thresholds low enough that many cells are
    accepted and lists go stale."""
    _check(synth.random_small(86000 + seed, max_side=48, max_n=120, max_depth=6, max_T=6), seed)


@pytest.mark.parametrize("k", range(2))
def test_model_matches_the_oracle_on_plain_128(k):
    _check(synth.plain_128(index=k), 1000 + k)


def test_list_order_changes_no_result():
    """The same image under several shuffles of every list gives one result."""
    img = synth.random_small(86500, max_side=40, max_n=100, max_depth=5, max_T=3)
    first = _walk_model(img.points, img.W, img.H, img.depth, img.T, random.Random(0))
    for s in range(1, 4):
        again = _walk_model(img.points, img.W, img.H, img.depth, img.T, random.Random(s))
        for a, b in zip(first, again):
            assert np.array_equal(a, b)
