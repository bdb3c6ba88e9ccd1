"""GPU parity of the front end (Section 3: Sobel's gradient operator and the
ALPHA/BETA split) and of detection on the split sets, against the oracle.

Edge lists are integer results: both sides emit them in row-major order, so
they must be equal element by element.  Detection on the split sets must
equal the oracle's split detection (ALPHA as half 0, BETA as half 1).
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


def _np(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def _edges_equal(ctx, g, on_device_input):
    import torch
    img = torch.from_numpy(g.pixels).cuda() if on_device_input else g.pixels
    a, b = ctx.edges(img, g.threshold)
    wa, wb = oracle.edges(g.pixels, g.threshold)
    assert np.array_equal(_np(a), wa), g.name
    assert np.array_equal(_np(b), wb), g.name


@pytest.mark.parametrize("k", range(2))
def test_edges_gray_256(ctx, k):
    _edges_equal(ctx, synth.gray_256(index=k), on_device_input=(k == 1))


@pytest.mark.parametrize("seed", range(24))
def test_edges_random_shapes(ctx, seed):
    # includes images narrower or lower than 3 pixels (no interior) and widths
    # below 8, where one thread's pixels span several rows
    g = synth.gray_random(5100 + seed, max_side=70 if seed % 3 else 9)
    _edges_equal(ctx, g, on_device_input=bool(seed % 2))


def test_edges_full_size_4096(ctx):
    _edges_equal(ctx, synth.gray_4096(), on_device_input=True)


def test_edges_thresholds_and_capacity(ctx, hht):
    g = synth.gray_256(index=3)
    lib = hht.load()
    for thr in (0, 1, 150, 1443, 1500, 100000):
        a, b = ctx.edges(g.pixels, thr)
        wa, wb = oracle.edges(g.pixels, thr)
        assert np.array_equal(_np(a), wa) and np.array_equal(_np(b), wb), thr
    # too small a buffer: nothing copied, the needed lengths reported
    na, nb = ctypes.c_uint64(), ctypes.c_uint64()
    small = np.full((2, 2), -7, np.int16)
    rc = lib.hht_edges(ctx._h, g.pixels.ctypes.data, g.W, g.H, g.threshold, small.ctypes.data, 2, ctypes.byref(na),
                       small.ctypes.data, 2, ctypes.byref(nb))
    wa, wb = oracle.edges(g.pixels, g.threshold)
    assert rc == hht.HHT_E_CAPACITY and (na.value, nb.value) == (len(wa), len(wb))
    assert (small == -7).all()
    with pytest.raises(hht.HhtError):
        ctx.edges(g.pixels, -1)


def _split_want(g):
    a, b = oracle.edges(g.pixels, g.threshold)
    return oracle.detect_split(a, b, g.W, g.H, g.depth, g.T)


@pytest.mark.parametrize("k", range(2))
def test_detect_image_gray_256(ctx, k):
    g = synth.gray_256(index=k)
    got = ctx.detect_image(g.pixels, g.threshold, g.depth, g.T)
    want = _split_want(g)
    assert np.array_equal(got.leaves_numpy(), want.leaves)
    assert np.array_equal(got.stats, want.stats)


@pytest.mark.parametrize("seed", range(12))
def test_detect_image_random(ctx, seed):
    g = synth.gray_random(5200 + seed, max_side=90)
    got = ctx.detect_image(g.pixels, g.threshold, g.depth, g.T)
    want = _split_want(g)
    assert np.array_equal(got.leaves_numpy(), want.leaves), g.name
    assert np.array_equal(got.stats, want.stats), g.name


def test_detect_image_4096_equals_halves_of_plain_detection(ctx):
    # full size: the split detection equals half 0 of detecting ALPHA alone and
    # half 1 of detecting BETA alone (plain detection is checked against the
    # oracle elsewhere); the edge lists themselves against the oracle
    g = synth.gray_4096()
    got = ctx.detect_image(g.pixels, g.threshold, g.depth, g.T)
    a, b = ctx.edges(g.pixels, g.threshold)
    wa, wb = oracle.edges(g.pixels, g.threshold)
    assert np.array_equal(_np(a), wa) and np.array_equal(_np(b), wb)
    ra = ctx.detect(a, g.W, g.H, g.depth, g.T)
    rb = ctx.detect(b, g.W, g.H, g.depth, g.T)
    la, lb = ra.leaves_numpy(), rb.leaves_numpy()
    want = np.concatenate([la[la[:, 0] == 0], lb[lb[:, 0] == 1]])
    assert np.array_equal(got.leaves_numpy(), want)
    assert np.array_equal(got.stats[0], ra.stats[0]) and np.array_equal(got.stats[1], rb.stats[1])


def test_detect_image_capacity_and_fetch(ctx, hht):
    g = synth.gray_256(index=2)
    want = _split_want(g)
    lib = hht.load()
    r = hht._Result()
    small = np.zeros((1, 4), np.int32)
    r.leaves = small.ctypes.data
    r.leaf_capacity = 1
    rc = lib.hht_detect_image(ctx._h, g.pixels.ctypes.data, g.W, g.H, g.threshold, g.depth, g.T, ctypes.byref(r))
    assert rc == hht.HHT_E_CAPACITY and r.n_leaves == len(want.leaves)
    full = np.zeros((int(r.n_leaves), 4), np.int32)
    assert lib.hht_fetch_leaves(ctx._h, 0, full.ctypes.data, len(full)) == hht.HHT_OK
    assert np.array_equal(full.astype(np.uint32), want.leaves)
