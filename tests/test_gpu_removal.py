"""GPU parity of the solution() traversal (Section 3: voters of an accepted
leaf are plotted and removed from every region visited later) against the
oracle's removal mode: accepted cells in visiting order, per-level
statistics and the plotted points, bit for bit."""
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


def _check(ctx, img):
    got, plotted = ctx.detect_removal(img.points, img.W, img.H, img.depth, img.T)
    want, want_plotted = oracle.detect_removal(img.points, img.W, img.H, img.depth, img.T)
    assert np.array_equal(got.leaves_numpy(), want.leaves), img.name
    assert np.array_equal(got.stats, want.stats), img.name
    assert np.array_equal(plotted, want_plotted), img.name


@pytest.mark.parametrize("k", range(3))
def test_removal_plain_128(ctx, k):
    _check(ctx, synth.plain_128(index=k))


@pytest.mark.parametrize("seed", range(20))
def test_removal_random_shapes(ctx, seed):
    _check(ctx, synth.random_small(83000 + seed, max_side=300, max_n=2500, max_depth=9, max_T=12))


def test_removal_plain_1024(ctx):
    _check(ctx, synth.plain_1024())


def test_removal_batch_and_edges(ctx, hht):
    imgs = [synth.plain_128(index=k) for k in range(2)] + [synth.batch_image(k) for k in (0, 1)] + \
        [synth.random_small(84000 + s, max_side=64, max_n=200, max_depth=6, max_T=3) for s in range(4)]
    res = ctx.detect_removal_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs])
    for im, r in zip(imgs, res):
        want, _ = oracle.detect_removal(im.points, im.W, im.H, im.depth, im.T)
        assert np.array_equal(r.leaves_numpy(), want.leaves), im.name
        assert np.array_equal(r.stats, want.stats), im.name
    img = synth.plain_128()
    none, plotted = ctx.detect_removal(img.points, img.W, img.H, img.depth, img.n + 1)
    assert none.n_leaves == 0 and plotted.sum() == 0
    empty, _ = ctx.detect_removal(np.zeros((0, 2), np.int16), 8, 8, 3, 1)
    assert empty.n_leaves == 0
    bad = img.points.copy()
    bad[3, 0] = img.W  # outside the image
    with pytest.raises(hht.HhtError) as e:
        ctx.detect_removal(bad, img.W, img.H, img.depth, img.T)
    assert e.value.code == hht.HHT_E_RANGE
