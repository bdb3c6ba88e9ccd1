"""hht_detect_noalloc: the detection entry point for callers that cannot let
the library allocate device memory (a process whose device memory belongs to
another framework's allocator, or a loop that cannot take the device-wide
synchronisation of an allocation).  Its scratch is one static device array
shared by every call, so it is checked here, in the file collected last,
through the C ABI: against the oracle and against the regular hht_detect
entry point, with identical leaves and statistics (the results are integers,
so the tolerance is exact equality), on two calls in a row; on a non-default
stream; and across a call that the array is too small for."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

_CAP = 1 << 18  # HHT_NOALLOC_MAX_LEAVES


@pytest.fixture(scope="module")
def lib():
    from paper_1007_0547_gb300 import build
    build.build()
    from paper_1007_0547_gb300 import hht
    lib = hht.load()
    lib.hht_detect_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.POINTER(hht._Result), ctypes.c_void_p]
    lib.hht_detect_noalloc.restype = ctypes.c_int
    return lib


def _stats(r, depth):
    return np.frombuffer(r.stats, dtype=np.uint64).reshape(2, 25, 4)[:, : depth + 1].copy()


def _regular(lib, pts, W, H, D, T):
    from paper_1007_0547_gb300 import hht
    ctx = ctypes.c_void_p()
    assert lib.hht_create(ctypes.byref(ctx), 0, None, 0) == hht.HHT_OK
    pts = np.ascontiguousarray(pts)
    leaves = np.zeros((_CAP, 4), np.uint32)
    r = hht._Result()
    r.leaves = leaves.ctypes.data
    r.leaf_capacity = _CAP
    assert lib.hht_detect(ctx, pts.ctypes.data, len(pts), W, H, D, T, ctypes.byref(r)) == hht.HHT_OK
    lib.hht_destroy(ctx)
    return leaves[: r.n_leaves].copy(), _stats(r, D)


def _noalloc(lib, pts, W, H, D, T, on_device, stream=None):
    """One call of hht_detect_noalloc; returns (rc, leaves, stats)."""
    import torch
    from paper_1007_0547_gb300 import hht
    pts = np.ascontiguousarray(pts)
    if on_device:
        dpts = torch.from_numpy(pts).cuda()
        buf = torch.zeros((_CAP, 4), dtype=torch.int32, device="cuda")
        pp, lp = dpts.data_ptr(), buf.data_ptr()
    else:
        buf = np.zeros((_CAP, 4), np.uint32)
        pp, lp = pts.ctypes.data, buf.ctypes.data
    r = hht._Result()
    sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    if stream is not None:
        torch.cuda.current_stream().synchronize()  # the inputs above were written on the current stream
    rc = lib.hht_detect_noalloc(pp, len(pts), W, H, D, T, lp, _CAP, ctypes.byref(r), sp)
    assert r.status == rc
    if rc != hht.HHT_OK:
        return rc, None, None
    lv = buf[: r.n_leaves]
    lv = lv.cpu().numpy().astype(np.uint32) if on_device else lv.copy()
    return rc, lv, _stats(r, D)


def _cases():
    img = synth.plain_1024()
    return [(im.name, im.points, im.W, im.H, im.depth, im.T) for im in
            (synth.plain_128(index=0), synth.plain_128(index=3),
             synth.random_small(777, max_side=200, max_n=1500, max_depth=8, max_T=6))] + [
        # the 1024 x 1024 image's points at depth 7: about 29 MB of voter
        # lists in the two live levels, 11 706 leaves (at its own depth 10 the
        # image has 549 434 leaves, beyond the entry point's leaf limit)
        ("plain_1024 at depth 7", img.points, img.W, img.H, 7, img.T)]


def test_noalloc_matches_oracle_and_detect_on_two_calls_in_a_row(lib):
    from paper_1007_0547_gb300 import hht
    for name, pts, W, H, D, T in _cases():
        want = oracle.detect(pts, W, H, D, T)
        reg_leaves, reg_stats = _regular(lib, pts, W, H, D, T)
        assert np.array_equal(reg_leaves, want.leaves) and np.array_equal(reg_stats, want.stats), name
        for call in range(2):  # the static scratch keeps the previous call's contents
            rc, got_leaves, got_stats = _noalloc(lib, pts, W, H, D, T, on_device=(call == 1))
            assert rc == hht.HHT_OK, (name, hht.strerror(rc))
            assert np.array_equal(got_leaves, want.leaves), (name, call)
            assert np.array_equal(got_stats, want.stats), (name, call)


def test_noalloc_on_a_non_default_stream(lib):
    import torch
    from paper_1007_0547_gb300 import hht
    img = synth.plain_128(index=5)
    want = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    s = torch.cuda.Stream()
    for on_device in (False, True):
        rc, lv, st = _noalloc(lib, img.points, img.W, img.H, img.depth, img.T, on_device, stream=s)
        assert rc == hht.HHT_OK
        assert np.array_equal(lv, want.leaves) and np.array_equal(st, want.stats)


def test_noalloc_voter_lists_beyond_the_array_then_exact_again(lib):
    """The 1024 x 1024 image at depth 9 with T = 400 keeps 4 299 leaves but
    writes a 72.5 MB voter list at level 7, more than the 64 MiB array: the
    call returns HHT_E_NOMEM.  At its own depth 10 and T = 64 both its voter
    lists and its 549 434 leaves are beyond the limits: HHT_E_NOMEM as well.
    A call after each is exact."""
    from paper_1007_0547_gb300 import hht
    big = synth.plain_1024()
    small = synth.plain_128(index=2)
    want = oracle.detect(small.points, small.W, small.H, small.depth, small.T)
    for D, T in ((9, 400), (big.depth, big.T)):
        rc, _, _ = _noalloc(lib, big.points, big.W, big.H, D, T, on_device=True)
        assert rc == hht.HHT_E_NOMEM, hht.strerror(rc)
        rc, lv, st = _noalloc(lib, small.points, small.W, small.H, small.depth, small.T, on_device=False)
        assert rc == hht.HHT_OK
        assert np.array_equal(lv, want.leaves) and np.array_equal(st, want.stats)


def test_noalloc_rejects_sizes_beyond_its_limits(lib):
    from paper_1007_0547_gb300 import hht
    r = hht._Result()
    pts = np.zeros((4, 2), np.int16)
    # depth beyond the stated maximum: refused before any device work
    assert lib.hht_detect_noalloc(pts.ctypes.data, 4, 8, 8, 17, 1, None, 0, ctypes.byref(r), None) == hht.HHT_E_NOMEM
    assert lib.hht_detect_noalloc(pts.ctypes.data, 4, 8, 8, 0, 1, None, 0, ctypes.byref(r), None) == hht.HHT_E_ARG
    # more points than the stated maximum
    many = np.zeros(((1 << 20) + 1, 2), np.int16)
    assert lib.hht_detect_noalloc(many.ctypes.data, len(many), 8, 8, 5, 1, None, 0, ctypes.byref(r),
                                  None) == hht.HHT_E_NOMEM
