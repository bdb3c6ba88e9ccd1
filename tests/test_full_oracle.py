"""CPU checks of the full-size oracle helper (tests/full_oracle.py): its
subtree shares, combined from the definitions, equal the whole oracle run,
and the thread pool gives the same results as one thread."""
import numpy as np
import pytest

import oracle
import synth
from tests import full_oracle


@pytest.mark.parametrize("split_level", [1, 2, 3])
def test_shares_combine_to_the_whole_detection(split_level):
    imgs = [synth.plain_128(index=3), synth.random_small(5150, max_side=200, max_n=900, max_depth=7, max_T=6),
            synth.batch_image(1)]
    with full_oracle.pool() as ex:
        for im in imgs:
            if im.depth < split_level:
                continue
            want = oracle.detect(im.points, im.W, im.H, im.depth, im.T)
            lv, st = full_oracle.detect(im.points, im.W, im.H, im.depth, im.T, split_level=split_level, ex=ex)
            assert np.array_equal(lv, want.leaves), (im.name, split_level)
            assert np.array_equal(st, want.stats), (im.name, split_level)


def test_share_masks_cover_every_region_once_in_depth_first_order():
    for k in (1, 2, 3):
        masks = full_oracle.share_masks(k)
        assert len(masks) == 2 * 4 ** k
        total = np.sum(masks, axis=0)
        assert (total == 1).all()
    # level 1, half 0: NE (a=1, b=1), NW (0, 1), SW (0, 0), SE (1, 0); then half 1
    first = [int(np.argmax(m)) for m in full_oracle.share_masks(1)]
    assert first == [3, 1, 0, 2, 7, 5, 4, 6]


def test_pool_matches_one_thread():
    imgs = [synth.plain_128(index=k) for k in range(4)] + [synth.batch_image(1)]
    with full_oracle.pool() as ex:
        futs = [ex.submit(full_oracle.detect, im.points, im.W, im.H, im.depth, im.T) for im in imgs]
        for im, f in zip(imgs, futs):
            lv, st = f.result()
            want = oracle.detect(im.points, im.W, im.H, im.depth, im.T)
            assert np.array_equal(lv, want.leaves) and np.array_equal(st, want.stats)
