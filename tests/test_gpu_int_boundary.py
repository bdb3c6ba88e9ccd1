"""GPU parity at the switch between 32-bit and 64-bit corner arithmetic.

The level kernels evaluate G(i, j) = 4L*j + 2x*i - 2LK - Kx - Ky (Section 2's
F scaled by K = 2^depth) in int32 when log2 L + depth <= 27 and in int64
above.  The int32 bound is tight at 27: |G| reaches 2^29 and the kernels'
intermediate x*A and (x + y)*K terms reach 2^28 each, largest for points at
the image's far corner.  Both sides of the switch are run here, 27 (int32)
and 28 (int64), on a large frame at a shallow depth (32767 x 32767, L = 2^15,
depths 12 and 13) and a small frame at a deep one (16 x 16, L = 2^4, depths
23 and 24), with points at all four image corners, lines through one grid
vertex (the concurrency case, where corners lie exactly on lines and the
tie rule decides) and scattered points; under the paper's 4-bit code and
under the prior-art circle test (built for int32 only: at 28 it is refused
with HHT_E_ARG before any device work).
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


def _points(side, seed):
    """Corners of the side x side image, collinear points on y = x/2 + c
    (parameter point m = 1/2, b = c, a grid vertex at these depths) and
    scattered points."""
    last = side - 1
    corners = [(0, 0), (last, 0), (0, last), (last, last)]
    c = 96 if side > 1000 else 2
    step = max(2, (side // 40) & ~1)
    line = [(x, x // 2 + c) for x in range(0, side, step) if x // 2 + c <= last]
    st = synth.Stream(seed)
    rnd = np.stack([st.ints(0, last, 24), st.ints(0, last, 24)], axis=1)
    pts = np.concatenate([np.array(corners + line), rnd]).astype(np.int16)
    return pts


CASES = [(32767, 12), (32767, 13), (16, 23), (16, 24)]


def _thresholds(side):
    # the 16 x 16 frame holds 8 collinear points; at depth 23-24 a threshold
    # of 2 would make every crossing of two lines a leaf (10^7-10^8 leaves)
    return (2, 6, 12) if side > 1000 else (3, 5, 8)


@pytest.mark.parametrize("side,depth", CASES)
def test_exact_code_on_both_sides_of_the_switch(hht, side, depth):
    pts = _points(side, 7000 + depth)
    ctx = hht.Context(device=0)
    try:
        for T in _thresholds(side):
            got = ctx.detect(pts, side, side, depth, T)
            want = oracle.detect(pts, side, side, depth, T)
            assert np.array_equal(got.leaves_numpy(), want.leaves), (side, depth, T)
            assert np.array_equal(got.stats, want.stats), (side, depth, T)
        # the vertex's neighbourhood reaches the leaf level
        assert len(want.leaves) > 0
    finally:
        ctx.close()


@pytest.mark.parametrize("side,depth", CASES)
def test_circle_test_on_both_sides_of_the_switch(hht, side, depth):
    pts = _points(side, 7100 + depth)
    ctx = hht.Context(device=0)
    try:
        ctx.set_predicate(hht.PREDICATE_FHT)
        lL = int(np.ceil(np.log2(side)))
        for T in _thresholds(side):
            if lL + depth > 27:
                with pytest.raises(hht.HhtError) as e:
                    ctx.detect(pts, side, side, depth, T)
                assert e.value.code == hht.HHT_E_ARG
                continue
            got = ctx.detect(pts, side, side, depth, T)
            want = oracle.detect(pts, side, side, depth, T, mode="fht")
            assert np.array_equal(got.leaves_numpy(), want.leaves), (side, depth, T)
            assert np.array_equal(got.stats, want.stats), (side, depth, T)
    finally:
        ctx.close()


@pytest.mark.parametrize("side,depth", CASES)
def test_batch_mixing_both_sides_of_the_switch(hht, side, depth):
    """A batch holding an image beyond the int32 bound runs every image of
    its wave in int64; the results of the small images are unchanged."""
    pts = _points(side, 7200 + depth)
    small = synth.plain_128(index=1)
    ctx = hht.Context(device=0)
    try:
        res = ctx.detect_batch([(pts, side, side, depth, 6), (small.points, 128, 128, small.depth, small.T)])
        for r, (p, W, D, T) in zip(res, [(pts, side, depth, 6), (small.points, 128, small.depth, small.T)]):
            want = oracle.detect(p, W, W, D, T)
            assert np.array_equal(r.leaves_numpy(), want.leaves) and np.array_equal(r.stats, want.stats)
    finally:
        ctx.close()


@pytest.mark.parametrize("side,depth", CASES)
def test_removal_on_both_sides_of_the_switch(hht, side, depth):
    """The solution() walk decides its children and grandchildren with the
    same corner signs, in int32 at 27 and int64 at 28."""
    pts = _points(side, 7100 + depth)
    ctx = hht.Context(device=0)
    try:
        for T in _thresholds(side):
            got, plotted = ctx.detect_removal(pts, side, side, depth, T)
            want, want_plotted = oracle.detect_removal(pts, side, side, depth, T)
            assert np.array_equal(got.leaves_numpy(), want.leaves), (side, depth, T)
            assert np.array_equal(got.stats, want.stats), (side, depth, T)
            assert np.array_equal(plotted, want_plotted), (side, depth, T)
    finally:
        ctx.close()
