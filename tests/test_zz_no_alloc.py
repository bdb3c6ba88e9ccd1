"""hht_detect_noalloc: the detection entry point for callers that cannot let
the library allocate device memory (stream capture, a foreign allocator,
latency-critical loops).  Its scratch is one static device array, so it is
checked here, in the file collected last, against the regular hht_detect
entry point through the C ABI: identical leaves and statistics (the results
are integers, so the tolerance is exact equality), on two calls in a row."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


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


def _regular(lib, img):
    from paper_1007_0547_gb300 import hht
    ctx = ctypes.c_void_p()
    assert lib.hht_create(ctypes.byref(ctx), 0, None, 0) == hht.HHT_OK
    pts = np.ascontiguousarray(img.points)
    cap = 1 << 18
    leaves = np.zeros((cap, 4), np.uint32)
    r = hht._Result()
    r.leaves = leaves.ctypes.data
    r.leaf_capacity = cap
    assert lib.hht_detect(ctx, pts.ctypes.data, img.n, img.W, img.H, img.depth, img.T, ctypes.byref(r)) == hht.HHT_OK
    lib.hht_destroy(ctx)
    st = np.frombuffer(r.stats, dtype=np.uint64).reshape(2, 25, 4)[:, : img.depth + 1].copy()
    return leaves[: r.n_leaves].copy(), st


def _noalloc(lib, img, on_device):
    import torch
    from paper_1007_0547_gb300 import hht
    cap = 1 << 18
    if on_device:
        pts = torch.from_numpy(np.ascontiguousarray(img.points)).cuda()
        buf = torch.zeros((cap, 4), dtype=torch.int32, device="cuda")
        pp, lp = pts.data_ptr(), buf.data_ptr()
    else:
        pts = np.ascontiguousarray(img.points)
        buf = np.zeros((cap, 4), np.uint32)
        pp, lp = pts.ctypes.data, buf.ctypes.data
    r = hht._Result()
    rc = lib.hht_detect_noalloc(pp, img.n, img.W, img.H, img.depth, img.T, lp, cap, ctypes.byref(r), None)
    assert rc == hht.HHT_OK, hht.strerror(rc)
    lv = buf[: r.n_leaves]
    lv = lv.cpu().numpy().astype(np.uint32) if on_device else lv.copy()
    st = np.frombuffer(r.stats, dtype=np.uint64).reshape(2, 25, 4)[:, : img.depth + 1].copy()
    return lv, st


def test_noalloc_matches_detect_on_two_calls_in_a_row(lib):
    imgs = [synth.plain_128(index=0), synth.plain_128(index=3),
            synth.random_small(777, max_side=200, max_n=1500, max_depth=8, max_T=6)]
    for img in imgs:
        want_leaves, want_stats = _regular(lib, img)
        for call in range(2):  # the static scratch keeps the previous call's contents
            got_leaves, got_stats = _noalloc(lib, img, on_device=(call == 1))
            assert np.array_equal(got_leaves, want_leaves), (img.name, call)
            assert np.array_equal(got_stats, want_stats), (img.name, call)


def test_noalloc_rejects_sizes_beyond_its_limits(lib):
    from paper_1007_0547_gb300 import hht
    r = hht._Result()
    pts = np.zeros((4, 2), np.int16)
    # depth beyond the stated maximum: refused before any device work
    assert lib.hht_detect_noalloc(pts.ctypes.data, 4, 8, 8, 17, 1, None, 0, ctypes.byref(r), None) == hht.HHT_E_NOMEM
    assert lib.hht_detect_noalloc(pts.ctypes.data, 4, 8, 8, 0, 1, None, 0, ctypes.byref(r), None) == hht.HHT_E_ARG
