"""Pins of the oracle's front end (Section 3: Sobel's gradient operator and the
ALPHA/BETA split) and of its split detection.

- hand-worked step edges (tests/golden/sobel_steps.json);
- Sobel's responses against scipy.ndimage.sobel (a library routine) on the
  interior pixels of random images;
- transposing an image swaps ALPHA and BETA (away from ties |gx| = |gy|);
- raising the threshold only removes edge points; threshold 0 keeps every
  interior pixel;
- split detection with every point in both sets is the plain detection.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sobel_steps.json")


def _pts(lst):
    return np.array(lst, dtype=np.int16).reshape(-1, 2)


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"][:30])
def test_hand_worked_steps(case):
    img = np.array(case["pixels"], dtype=np.uint8)
    assert img.shape == (case["H"], case["W"])
    a, b = oracle.edges(img, case["threshold"])
    assert np.array_equal(a, _pts(case["alpha"]))
    assert np.array_equal(b, _pts(case["beta"]))


def test_sobel_against_scipy():
    ndimage = pytest.importorskip("scipy.ndimage")
    st = synth.Stream(404)
    for _ in range(6):
        W, H = (int(v) for v in st.ints(3, 40, 2))
        img = st.ints(0, 255, W * H).astype(np.uint8).reshape(H, W)
        f = img.astype(np.int64)
        sx = ndimage.sobel(f, axis=1)  # derivative along x (columns), smoothed along y
        sy = ndimage.sobel(f, axis=0)
        for y in range(1, H - 1):
            for x in range(1, W - 1):
                assert oracle.sobel(img, x, y) == (int(sx[y, x]), int(sy[y, x])), (x, y)


def test_edges_follow_gradients_and_row_major_order():
    g = synth.gray_random(17, max_side=48)
    a, b = oracle.edges(g.pixels, g.threshold)
    for pts, want_alpha in ((a, True), (b, False)):
        key = pts[:, 1].astype(np.int64) * g.W + pts[:, 0]
        assert np.all(np.diff(key) > 0)
        for x, y in pts:
            gx, gy = oracle.sobel(g.pixels, int(x), int(y))
            assert gx * gx + gy * gy >= g.threshold ** 2
            assert (abs(gx) <= abs(gy)) == want_alpha


def test_transpose_swaps_alpha_and_beta_away_from_ties():
    g = synth.gray_256()
    a, b = oracle.edges(g.pixels, g.threshold)
    at, bt = oracle.edges(np.ascontiguousarray(g.pixels.T), g.threshold)

    def untied(pts, img):
        keep = []
        for x, y in pts:
            gx, gy = oracle.sobel(img, int(x), int(y))
            if abs(gx) != abs(gy):
                keep.append((int(x), int(y)))
        return set(keep)

    assert untied(a, g.pixels) == {(y, x) for x, y in untied(bt, g.pixels.T)}
    assert untied(b, g.pixels) == {(y, x) for x, y in untied(at, g.pixels.T)}


def test_threshold_monotone_and_zero_keeps_interior():
    g = synth.gray_random(23, max_side=40)
    prev = None
    for thr in (0, 50, 150, 400, 2000):
        a, b = oracle.edges(g.pixels, thr)
        s = {tuple(p) for p in a.tolist()} | {tuple(p) for p in b.tolist()}
        if thr == 0:
            assert len(s) == max(0, g.W - 2) * max(0, g.H - 2)
        if prev is not None:
            assert s <= prev
        prev = s


def test_split_detection_with_both_sets_full_is_plain_detection():
    img = synth.plain_128(index=2)
    both = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    split = oracle.detect_split(img.points, img.points, img.W, img.H, img.depth, img.T)
    assert np.array_equal(split.leaves, both.leaves)
    assert np.array_equal(split.stats, both.stats)
