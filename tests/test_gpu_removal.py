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


@pytest.mark.parametrize("k", [13, 160])
def test_removal_heaviest_batch_images(ctx, k):
    """Two of the batch's slowest walks at full size (sides 2021 and 2023,
    depth 11): many accepted cells, so children's lists go stale at every
    depth and the leaves' counts taken two levels up are often overruled."""
    _check(ctx, synth.batch_image(k))


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


# ------------------------------------------------------------------ the plotted points as a raster
def _scatter(points, W, H, plotted):
    """The oracle's plotted flags scattered to their pixels: bit h for half h."""
    r = np.zeros((H, W), np.uint8)
    pts = np.asarray(points, np.int64).reshape(-1, 2)
    for h in (0, 1):
        sel = plotted[h].astype(bool)
        r[pts[sel, 1], pts[sel, 0]] |= np.uint8(1 << h)
    return r


def test_raster_equals_scatter_of_oracle_flags(ctx):
    imgs = [synth.plain_128(index=k) for k in range(3)] + [synth.plain_1024()] + \
        [synth.random_small(85000 + s, max_side=120, max_n=2500, max_depth=8, max_T=6) for s in range(6)]
    for im in imgs:
        ctx.detect_removal(im.points, im.W, im.H, im.depth, im.T, with_plotted=False)
        _, want_plotted = oracle.detect_removal(im.points, im.W, im.H, im.depth, im.T)
        want = _scatter(im.points, im.W, im.H, want_plotted)
        host = ctx.removal_raster(0, im.W, im.H)
        dev = ctx.removal_raster(0, im.W, im.H, on_device=True).cpu().numpy()
        assert np.array_equal(host, want), im.name
        assert np.array_equal(dev, want), im.name


def test_raster_of_each_image_of_a_batch(ctx, hht):
    imgs = [synth.plain_128(index=3), synth.batch_image(2), synth.random_small(86000, max_side=90, max_n=800,
                                                                              max_depth=7, max_T=4)]
    ctx.detect_removal_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs])
    for k, im in enumerate(imgs):
        _, want_plotted = oracle.detect_removal(im.points, im.W, im.H, im.depth, im.T)
        assert np.array_equal(ctx.removal_raster(k, im.W, im.H), _scatter(im.points, im.W, im.H, want_plotted))
    with pytest.raises(hht.HhtError) as e:
        ctx.removal_raster(len(imgs), 8, 8)
    assert e.value.code == hht.HHT_E_ARG
    # a removal job that failed leaves nothing to draw
    bad = imgs[0].points.copy()
    bad[0, 0] = imgs[0].W
    with pytest.raises(hht.HhtError):
        ctx.detect_removal(bad, imgs[0].W, imgs[0].H, imgs[0].depth, imgs[0].T)
    with pytest.raises(hht.HhtError) as e:
        ctx.removal_raster(0, imgs[0].W, imgs[0].H)
    assert e.value.code == hht.HHT_E_ARG


def test_plotted_flags_into_device_memory(ctx, hht):
    """The plotted flags are expanded on the device, into a device buffer
    directly or through a staging buffer into host memory."""
    import ctypes
    import torch
    im = synth.plain_128(index=4)
    want_res, want_plotted = oracle.detect_removal(im.points, im.W, im.H, im.depth, im.T)
    lib = hht.load()
    leaves = np.zeros((2 * (im.n // im.T + 1), 4), np.int32)
    flags = torch.full((2, im.n), 7, dtype=torch.uint8, device="cuda")
    r = hht._Result()
    r.leaves = leaves.ctypes.data
    r.leaf_capacity = len(leaves)
    pts = np.ascontiguousarray(im.points)
    assert lib.hht_detect_removal(ctx._h, pts.ctypes.data, im.n, im.W, im.H, im.depth, im.T, ctypes.byref(r),
                                  flags.data_ptr()) == hht.HHT_OK
    assert np.array_equal(flags.cpu().numpy(), want_plotted)
    assert np.array_equal(leaves[: r.n_leaves].astype(np.uint32), want_res.leaves)
