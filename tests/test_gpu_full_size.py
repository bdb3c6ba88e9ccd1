"""Full-size GPU parity: every leaf and every statistic of the 256-image mixed
batch and of the 4096 x 4096 image, element by element against the oracle.

The GPU runs each workload exactly as the benchmark does (the batch in one
detect_batch call, in the context's default tile shape).  The oracle runs on
all host cores (tests/full_oracle.py): the batch one image per thread, the
4096 x 4096 image as 128 level-3 subtree shares.  Results are integers decided
by exact comparisons, so the check is bit-exact: the leaves (half, i, j, votes)
in depth-first order and stats[half, level] = (tested, passed, votes, tests).
"""
import time

import numpy as np
import pytest

import synth
from tests import full_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hht():
    from paper_1007_0547_gb300 import build
    build.build()
    from paper_1007_0547_gb300 import hht as mod
    return mod


def _mismatch(name, got_leaves, got_stats, want_leaves, want_stats):
    """None when equal, else a short description of the first difference."""
    if not np.array_equal(got_stats, want_stats):
        bad = np.argwhere(got_stats != want_stats)[0]
        return f"{name}: stats[{tuple(bad)}] gpu {got_stats[tuple(bad)]} oracle {want_stats[tuple(bad)]}"
    if got_leaves.shape != want_leaves.shape:
        return f"{name}: {len(got_leaves)} leaves on the gpu, {len(want_leaves)} from the oracle"
    if not np.array_equal(got_leaves, want_leaves):
        k = int(np.argwhere((got_leaves != want_leaves).any(axis=1))[0, 0])
        return f"{name}: leaf {k} gpu {got_leaves[k].tolist()} oracle {want_leaves[k].tolist()}"
    return None


def test_batch_256_every_image_every_leaf(hht):
    """All 256 images of the mixed batch (sides 256-2048, depths 8-11, about
    2.1e11 line x region tests and 2.1e8 leaves) against the oracle."""
    imgs = synth.batch_256()
    ctx = hht.Context(device=0)
    try:
        res = ctx.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs], leaves_on_device=False)
    finally:
        ctx.close()
    got = {k: (r.leaves_numpy(), r.stats) for k, r in enumerate(res)}
    del res
    # largest oracle runs first, so that the pool finishes together
    order = sorted(range(len(imgs)), key=lambda k: -imgs[k].n * (1 << imgs[k].depth))
    errors, t0, leaves_checked = [], time.time(), 0
    with full_oracle.pool() as ex:
        futs = {ex.submit(full_oracle.detect, imgs[k].points, imgs[k].W, imgs[k].H, imgs[k].depth, imgs[k].T): k
                for k in order}
        for f in list(futs):
            k = futs.pop(f)
            lv, st = f.result()
            g_lv, g_st = got.pop(k)
            e = _mismatch(imgs[k].name, g_lv, g_st, lv, st)
            if e:
                errors.append(e)
            leaves_checked += len(lv)
    print(f"batch_256: {leaves_checked} leaves of 256 images checked in {time.time() - t0:.1f} s")
    assert not errors, errors[:5]


def test_plain_4096_every_leaf(hht):
    """The 4096 x 4096 image (about 7.1e5 points, depth 12, T = 128; about
    1.1e7 leaves) against the oracle run as 128 level-3 subtree shares."""
    img = synth.plain_4096()
    ctx = hht.Context(device=0)
    try:
        r = ctx.detect(img.points, img.W, img.H, img.depth, img.T, leaves_on_device=False)
        g_lv, g_st = r.leaves_numpy(), r.stats
    finally:
        ctx.close()
    t0 = time.time()
    lv, st = full_oracle.detect(img.points, img.W, img.H, img.depth, img.T, split_level=3)
    print(f"plain_4096: {len(lv)} leaves checked in {time.time() - t0:.1f} s")
    e = _mismatch(img.name, g_lv, g_st, lv, st)
    assert e is None, e
