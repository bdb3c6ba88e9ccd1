"""Failure path on the GPU, made without a GPU fault.

Host-side fault injection (hht_inject_fault) withholds one tile of the
selection's look-back scan: that tile publishes nothing, so the tiles after it
wait on a flag that nothing sets.  Every such wait is bounded, so the job must
come back with HHT_E_TIMEOUT within seconds, and the same context must then
give the same results as before the fault (checked against the oracle).
"""
import time

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


def _dev(img):
    import torch
    return torch.from_numpy(img.points).to("cuda:0")


def test_withheld_scan_tile_times_out_and_the_context_recovers(hht):
    # 1024 x 1024: the deep levels hold tens of thousands of regions, i.e.
    # several selection tiles of 1024 parents, so tile 0's successors wait
    big, small = synth.plain_1024(), synth.plain_128()
    ctx = hht.Context(device=0)
    try:
        before = ctx.detect(_dev(big), big.W, big.H, big.depth, big.T)
        lv_before = before.leaves_numpy().copy()
        ctx.inject_fault(hht.FAULT_WITHHOLD_SCAN_TILE, 0)
        t0 = time.perf_counter()
        with pytest.raises(hht.HhtError) as err:
            ctx.detect(_dev(big), big.W, big.H, big.depth, big.T)
        waited = time.perf_counter() - t0
        assert err.value.code == hht.HHT_E_TIMEOUT
        assert waited < 60.0, f"the bounded waits took {waited:.1f} s"
        # the injection lasted one job: the context works as before
        after = ctx.detect(_dev(big), big.W, big.H, big.depth, big.T)
        assert np.array_equal(after.leaves_numpy(), lv_before)
        assert np.array_equal(after.stats, before.stats)
        got = ctx.detect(_dev(small), small.W, small.H, small.depth, small.T)
        want = oracle.detect(small.points, small.W, small.H, small.depth, small.T)
        assert np.array_equal(got.leaves_numpy(), want.leaves)
        assert np.array_equal(got.stats, want.stats)
    finally:
        ctx.close()


def test_withheld_tile_in_a_batch_fails_the_batch_only_once(hht):
    imgs = [synth.plain_1024(index=1)] + [synth.plain_128(index=k) for k in range(3)]
    batch = [(_dev(im), im.W, im.H, im.depth, im.T) for im in imgs]
    ctx = hht.Context(device=0)
    try:
        ref = ctx.detect_batch(batch)
        ref_leaves = [r.leaves_numpy().copy() for r in ref]
        ctx.inject_fault(hht.FAULT_WITHHOLD_SCAN_TILE, 1)
        with pytest.raises(hht.HhtError) as err:
            ctx.detect_batch(batch)
        assert err.value.code == hht.HHT_E_TIMEOUT
        again = ctx.detect_batch(batch)
        for r, lv, r0 in zip(again, ref_leaves, ref):
            assert np.array_equal(r.leaves_numpy(), lv)
            assert np.array_equal(r.stats, r0.stats)
        want = oracle.detect(imgs[1].points, imgs[1].W, imgs[1].H, imgs[1].depth, imgs[1].T)
        assert np.array_equal(again[1].leaves_numpy(), want.leaves)
    finally:
        ctx.close()


def test_injection_beyond_the_last_tile_changes_nothing(hht):
    img = synth.plain_128()
    ctx = hht.Context(device=0)
    try:
        ctx.inject_fault(hht.FAULT_WITHHOLD_SCAN_TILE, 1 << 30)  # no selection has that many tiles
        got = ctx.detect(_dev(img), img.W, img.H, img.depth, img.T)
        want = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
        assert np.array_equal(got.leaves_numpy(), want.leaves)
        ctx.inject_fault(hht.FAULT_WITHHOLD_SCAN_TILE, 0)
        ctx.inject_fault(hht.FAULT_NONE)  # cleared before any job ran
        got = ctx.detect(_dev(img), img.W, img.H, img.depth, img.T)
        assert np.array_equal(got.stats, want.stats)
        with pytest.raises(hht.HhtError):
            ctx.inject_fault(7)
    finally:
        ctx.close()
