"""GPU parity of the prior-art FHT circle test (the paper's comparison method,
Sections 1 and 3, Table 1) against the oracle's FHT mode.

The circle test is decided exactly on integers on both sides, so leaves (in
depth-first order) and per-level statistics must agree bit for bit.  The
relation to the exact test is checked on the GPU output too: every region's
exact voters are circle voters, so exact leaves are FHT leaves with no more
votes, and the FHT never casts fewer votes (C_v >= 1).
"""
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
def fctx(hht):
    c = hht.Context(device=0)
    c.set_predicate(hht.PREDICATE_FHT)
    yield c
    c.close()


def _same_fht(got, img):
    want = oracle.detect(img.points, img.W, img.H, img.depth, img.T, mode="fht")
    g = got.leaves_numpy()
    assert g.shape == want.leaves.shape, (img.name, g.shape, want.leaves.shape)
    assert np.array_equal(g, want.leaves), img.name
    assert np.array_equal(got.stats, want.stats), img.name
    return want


@pytest.mark.parametrize("k", range(3))
def test_fht_plain_128(fctx, k):
    img = synth.plain_128(index=k)
    _same_fht(fctx.detect(img.points, img.W, img.H, img.depth, img.T), img)


@pytest.mark.parametrize("seed", range(24))
def test_fht_random_shapes(fctx, seed):
    img = synth.random_small(91000 + seed, max_side=300, max_n=2500, max_depth=9, max_T=12)
    _same_fht(fctx.detect(img.points, img.W, img.H, img.depth, img.T), img)


def test_fht_batch_of_mixed_images(fctx):
    imgs = [synth.random_small(92000 + s, max_side=400, max_n=3000, max_depth=9, max_T=30) for s in range(10)]
    imgs += [synth.plain_128(index=3)]
    res = fctx.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs])
    for im, r in zip(imgs, res):
        _same_fht(r, im)


def test_fht_against_exact_on_the_gpu(hht, fctx):
    import torch
    img = synth.plain_1024()
    pts = torch.from_numpy(img.points).cuda()
    ectx = hht.Context(device=0)
    try:
        ex = ectx.detect(pts, img.W, img.H, img.depth, img.T)
    finally:
        ectx.close()
    fh = fctx.detect(pts, img.W, img.H, img.depth, img.T)
    el, fl = ex.leaves_numpy().astype(np.int64), fh.leaves_numpy().astype(np.int64)
    fmap = {(h, i, j): v for h, i, j, v in fl}
    for h, i, j, v in el:
        assert fmap.get((h, i, j), -1) >= v, (h, i, j)
    assert fh.stats[:, :, 2].sum() >= ex.stats[:, :, 2].sum()  # C_v >= 1
    # sampled FHT leaves recounted over all points with the oracle's circle test
    rng = np.random.default_rng(5)
    for idx in rng.choice(len(fl), size=6, replace=False):
        h, i, j, v = (int(t) for t in fl[idx])
        L = oracle.frame_side(img.W, img.H)
        cnt = 0
        for x, y in img.points:
            px, py = (int(x), int(y)) if h == 0 else (int(y), int(x))
            cnt += oracle.fht_votes(px, py, i, j, 1, L, img.depth)
        assert cnt == v, (h, i, j)


def test_fht_size_limit_and_switching_back(hht):
    ctx = hht.Context(device=0)
    try:
        ctx.set_predicate(hht.PREDICATE_FHT)
        pts = np.zeros((1, 2), np.int16)
        with pytest.raises(hht.HhtError) as e:
            ctx.detect(pts, 32767, 32767, 13, 1)  # log2 L + depth = 28: outside the int32 build
        assert e.value.code == hht.HHT_E_ARG
        img = synth.plain_128(index=1)
        fh = ctx.detect(img.points, img.W, img.H, img.depth, img.T)
        ctx.set_predicate(hht.PREDICATE_EXACT)
        ex = ctx.detect(img.points, img.W, img.H, img.depth, img.T)
        want = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
        assert np.array_equal(ex.leaves_numpy(), want.leaves)
        assert np.array_equal(ex.stats, want.stats)
        assert fh.stats[:, :, 2].sum() >= ex.stats[:, :, 2].sum()
        with pytest.raises(hht.HhtError):
            ctx.set_predicate(5)
    finally:
        ctx.close()
