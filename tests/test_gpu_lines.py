"""GPU parity of the leaf -> line step (hht_lines) against the oracle.

Lines are integer results (peak leaf, cell count, vote total, exact centre
sums) in a fixed order (each cluster's first leaf), so they must be equal
element by element.  The oracle's clustering is quadratic, so full-size
images are checked against scipy.ndimage.label (a library routine) on the
dense K x K grid of each half, with 8-connectivity.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hht():
    from paper_1007_0547_gb300 import build
    build.build()
    from paper_1007_0547_gb300 import hht as mod
    return mod


@pytest.fixture(scope="module")
def ctx(hht):
    c = hht.Context(device=0)
    yield c
    c.close()


def _rows(a):
    return [(int(r["half"]), int(r["i"]), int(r["j"]), int(r["votes"]), int(r["cells"]), int(r["total_votes"]),
             int(r["sum_i2"]), int(r["sum_j2"])) for r in a]


def _label_check(lines, leaves, depth):
    ndimage = pytest.importorskip("scipy.ndimage")
    K = 1 << depth
    want = []
    for h in (0, 1):
        sel = np.nonzero(leaves[:, 0] == h)[0]
        grid = np.zeros((K, K), dtype=bool)
        grid[leaves[sel, 1], leaves[sel, 2]] = True
        lab, _ = ndimage.label(grid, structure=np.ones((3, 3), dtype=int))
        comp = lab[leaves[sel, 1], leaves[sel, 2]]
        for c in np.unique(comp):
            members = sel[comp == c]
            v = leaves[members, 3].astype(np.int64)
            peak = members[np.lexsort((members, -v))[0]]
            want.append((int(members.min()), (h, int(leaves[peak, 1]), int(leaves[peak, 2]), int(leaves[peak, 3]),
                                              len(members), int(v.sum()),
                                              int((v * (2 * leaves[members, 1].astype(np.int64) + 1)).sum()),
                                              int((v * (2 * leaves[members, 2].astype(np.int64) + 1)).sum()))))
    want.sort()
    assert _rows(lines) == [w for _, w in want]


@pytest.mark.parametrize("k", range(3))
def test_lines_plain_128(ctx, k):
    img = synth.plain_128(index=k)
    res = ctx.detect(img.points, img.W, img.H, img.depth, img.T)
    want = oracle.lines(oracle.detect(img.points, img.W, img.H, img.depth, img.T).leaves)
    got = ctx.lines(0)
    assert [r[:6] + (r[6], r[7]) for r in _rows(got)] == [
        (int(r["half"]), int(r["i"]), int(r["j"]), int(r["votes"]), int(r["cells"]), int(r["total_votes"]),
         int(r["sum_i2"]), int(r["sum_j2"])) for r in want]
    assert int(got["cells"].sum()) == res.n_leaves


@pytest.mark.parametrize("seed", range(12))
def test_lines_random_small(ctx, seed):
    img = synth.random_small(61000 + seed, max_side=200, max_n=1500, max_depth=8, max_T=10)
    ctx.detect(img.points, img.W, img.H, img.depth, img.T)
    want = oracle.lines(oracle.detect(img.points, img.W, img.H, img.depth, img.T).leaves)
    assert _rows(ctx.lines(0)) == _rows(want)


def test_lines_full_size_1024_against_scipy_label(ctx):
    img = synth.plain_1024()
    res = ctx.detect(img.points, img.W, img.H, img.depth, img.T)
    _label_check(ctx.lines(0), res.leaves_numpy().astype(np.int64), img.depth)


def test_lines_of_batch_images_and_of_the_front_end(ctx):
    imgs = [synth.batch_image(k) for k in (0, 5)]
    res = ctx.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs])
    for k, (im, r) in enumerate(zip(imgs, res)):
        _label_check(ctx.lines(k), r.leaves_numpy().astype(np.int64), im.depth)
    g = synth.gray_256()
    r = ctx.detect_image(g.pixels, g.threshold, g.depth, g.T)
    _label_check(ctx.lines(0), r.leaves_numpy().astype(np.int64), g.depth)


def test_lines_empty_and_capacity(ctx, hht):
    img = synth.plain_128()
    ctx.detect(img.points, img.W, img.H, img.depth, 10 ** 6)  # T above n: no leaves
    assert len(ctx.lines(0)) == 0
    ctx.detect(img.points, img.W, img.H, img.depth, img.T)
    lib = hht.load()
    n = ctypes.c_uint64()
    small = np.zeros(1, dtype=hht.LINE_DTYPE)
    assert lib.hht_lines(ctx._h, 0, small.ctypes.data, 1, ctypes.byref(n)) == hht.HHT_E_CAPACITY
    assert n.value == len(oracle.lines(oracle.detect(img.points, img.W, img.H, img.depth, img.T).leaves))
    assert lib.hht_lines(ctx._h, 1, small.ctypes.data, 1, ctypes.byref(n)) == hht.HHT_E_ARG


def test_lines_second_call_copies_and_new_job_recomputes(ctx, hht):
    a, b = synth.plain_128(index=1), synth.plain_128(index=2)
    lib = hht.load()
    n = ctypes.c_uint64()
    for img in (a, b, a):
        ctx.detect(img.points, img.W, img.H, img.depth, img.T)
        assert lib.hht_lines(ctx._h, 0, None, 0, ctypes.byref(n)) == hht.HHT_E_CAPACITY
        buf = np.zeros(int(n.value), dtype=hht.LINE_DTYPE)
        assert lib.hht_lines(ctx._h, 0, buf.ctypes.data, len(buf), ctypes.byref(n)) == hht.HHT_OK
        want = oracle.lines(oracle.detect(img.points, img.W, img.H, img.depth, img.T).leaves)
        assert _rows(buf) == _rows(want)
