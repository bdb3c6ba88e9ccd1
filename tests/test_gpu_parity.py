"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Results are integers decided by exact comparisons, so every check is
bit-exact: the leaves (half, i, j, votes) in the order both sides emit them
(the paper's depth-first order) and the per-level statistics (tested, passed,
votes, tests) of both halves.  Full-size workloads, where the
oracle would take minutes, are checked on sampled cells counted directly by
the oracle, on the statistics of the levels a shallower oracle run reaches
(a region's fate at level l does not depend on the depth below it), and on
properties that hold at any size.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import pins

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


def _same(got, want):
    g = got.leaves_numpy()
    assert g.shape == want.leaves.shape, (g.shape, want.leaves.shape)
    assert np.array_equal(g, want.leaves)
    assert np.array_equal(got.stats, want.stats)


def _props(res, T, depth):
    lv = res.leaves_numpy().astype(np.int64)
    if len(lv):
        key = pins.dfs_keys(lv, depth)
        assert np.all(np.diff(key) > 0), "leaves unique and in depth-first order, half 0 first"
        assert np.all(lv[:, 3] >= T)
        assert np.all(lv[:, 1] < (1 << depth)) and np.all(lv[:, 2] < (1 << depth))
    st = res.stats.astype(np.int64)
    for h in (0, 1):
        assert st[h, 0, 0] == 1 and st[h, 0, 1] == 1
        for l in range(1, depth + 1):
            assert st[h, l, 0] == 4 * st[h, l - 1, 1]
            assert st[h, l, 2] >= T * st[h, l, 1]
        assert st[h, depth, 1] == int((lv[:, 0] == h).sum()) if len(lv) else st[h, depth, 1] == 0


def _sampled_cells(points, W, H, depth, res, k=24, seed=0):
    lv = res.leaves_numpy()
    if len(lv) == 0:
        return
    rng = np.random.default_rng(seed)
    for idx in rng.choice(len(lv), size=min(k, len(lv)), replace=False):
        h, i, j, v = (int(t) for t in lv[idx])
        assert oracle.count_region(points, W, H, depth, h, i, j, 1) == v, (h, i, j)


# ------------------------------------------------------------------ small and plain configs
@pytest.mark.parametrize("k", range(4))
def test_plain_128(ctx, k):
    img = synth.plain_128(index=k)
    _same(ctx.detect(img.points, img.W, img.H, img.depth, img.T),
          oracle.detect(img.points, img.W, img.H, img.depth, img.T))


def test_plain_1024(ctx):
    img = synth.plain_1024()
    got = ctx.detect(img.points, img.W, img.H, img.depth, img.T)
    _same(got, oracle.detect(img.points, img.W, img.H, img.depth, img.T))


@pytest.mark.parametrize("seed", range(48))
def test_random_shapes(ctx, seed):
    img = synth.random_small(20000 + seed, max_side=300, max_n=600, max_depth=9, max_T=12)
    _same(ctx.detect(img.points, img.W, img.H, img.depth, img.T),
          oracle.detect(img.points, img.W, img.H, img.depth, img.T))


@pytest.mark.parametrize("seed", range(6))
def test_dense_small_images(ctx, seed):
    # many points on few cells: long voter lists, many tiles, ragged tails
    st = synth.Stream(300 + seed)
    W = int(st.ints(40, 200, 1)[0])
    H = int(st.ints(40, 200, 1)[0])
    n = int(st.ints(2000, 9000, 1)[0])
    pts = np.stack([st.ints(0, W - 1, n), st.ints(0, H - 1, n)], axis=1).astype(np.int16)
    D = int(st.ints(5, 9, 1)[0])
    T = int(st.ints(1, 40, 1)[0])
    _same(ctx.detect(pts, W, H, D, T), oracle.detect(pts, W, H, D, T))


# ------------------------------------------------------------------ edge cases
def test_empty_and_single_point(ctx):
    r = ctx.detect(np.zeros((0, 2), np.int16), 64, 32, 5, 1)
    _same(r, oracle.detect(np.zeros((0, 2), np.int16), 64, 32, 5, 1))
    p = np.array([[17, 3]], np.int16)
    _same(ctx.detect(p, 64, 32, 6, 1), oracle.detect(p, 64, 32, 6, 1))


def test_threshold_above_n_and_depth_one(ctx):
    img = synth.plain_128(index=5)
    _same(ctx.detect(img.points, 128, 128, 7, img.n + 1), oracle.detect(img.points, 128, 128, 7, img.n + 1))
    for T in (1, 50, img.n):
        _same(ctx.detect(img.points, 128, 128, 1, T), oracle.detect(img.points, 128, 128, 1, T))


def test_one_pixel_image_and_thin_images(ctx):
    p = np.zeros((5, 2), np.int16)
    _same(ctx.detect(p, 1, 1, 3, 2), oracle.detect(p, 1, 1, 3, 2))
    st = synth.Stream(8)
    for W, H in [(1, 300), (300, 1), (3, 77)]:
        pts = np.stack([st.ints(0, W - 1, 200), st.ints(0, H - 1, 200)], axis=1).astype(np.int16)
        _same(ctx.detect(pts, W, H, 7, 3), oracle.detect(pts, W, H, 7, 3))


def test_int64_corner_arithmetic(ctx):
    # L * K beyond 2^27 selects the 64-bit corner path
    st = synth.Stream(12)
    pts = np.stack([st.ints(0, 32766, 300), st.ints(0, 32766, 300)], axis=1).astype(np.int16)
    _same(ctx.detect(pts, 32767, 32767, 13, 3), oracle.detect(pts, 32767, 32767, 13, 3))
    pts2 = np.stack([st.ints(0, 15, 60), st.ints(0, 15, 60)], axis=1).astype(np.int16)
    _same(ctx.detect(pts2, 16, 16, 24, 4), oracle.detect(pts2, 16, 16, 24, 4))


def test_largest_frame_and_depth(ctx):
    # 32767 x 32767 at depth 24 (corner values up to 2^41): lines meeting at a
    # grid vertex, so that the hierarchy reaches the leaf level around it
    xs = [0, 2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 22, 30000, 32766]
    pts = np.array([[x, x // 2 + 100] for x in xs], np.int16)
    for T in (13, 14, 15):
        _same(ctx.detect(pts, 32767, 32767, 24, T), oracle.detect(pts, 32767, 32767, 24, T))


def test_range_error_and_bad_arguments(ctx, hht):
    with pytest.raises(hht.HhtError) as e:
        ctx.detect(np.array([[3, 64]], np.int16), 64, 64, 5, 1)
    assert e.value.code == hht.HHT_E_RANGE
    for args in [(64, 64, 0, 1), (64, 64, 25, 1), (0, 64, 5, 1), (64, 64, 5, 0)]:
        with pytest.raises(hht.HhtError) as e:
            ctx.detect(np.array([[3, 4]], np.int16), *args)
        assert e.value.code == hht.HHT_E_ARG
    # the context still works afterwards
    img = synth.plain_128()
    _same(ctx.detect(img.points, img.W, img.H, img.depth, img.T),
          oracle.detect(img.points, img.W, img.H, img.depth, img.T))


def test_host_and_device_inputs_and_outputs(ctx):
    import torch
    img = synth.plain_128(index=2)
    want = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    dev = torch.from_numpy(img.points).cuda()
    _same(ctx.detect(dev, img.W, img.H, img.depth, img.T), want)
    _same(ctx.detect(img.points, img.W, img.H, img.depth, img.T, leaves_on_device=False), want)
    _same(ctx.detect(dev, img.W, img.H, img.depth, img.T, leaves_on_device=False), want)


def test_caller_leaf_buffers_pinned_and_device(ctx):
    import torch
    imgs = [synth.plain_128(index=k) for k in range(3)] + [synth.random_small(777, max_side=300, max_n=2000,
                                                                              max_depth=8, max_T=10)]
    want = [oracle.detect(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
    total = sum(len(w.leaves) for w in want)
    batch = [(torch.from_numpy(im.points).pin_memory(), im.W, im.H, im.depth, im.T) for im in imgs]
    for out in (torch.full((total + 5, 4), -1, dtype=torch.int32).pin_memory(),
                torch.full((total, 4), -1, dtype=torch.int32, device="cuda"),
                np.full((total + 1, 4), -1, np.int32)):
        res = ctx.detect_batch(batch, leaves_out=out)
        for r, w in zip(res, want):
            _same(r, w)
        host = out.cpu().numpy() if isinstance(out, torch.Tensor) else out
        # the buffer holds every image's leaves (each result is a view at its
        # image's offset) and nothing past them
        got_rows = np.sort(host[:total].astype(np.uint32).view(np.dtype((np.void, 16))).ravel())
        want_rows = np.sort(np.ascontiguousarray(np.concatenate([w.leaves for w in want])).view(
            np.dtype((np.void, 16))).ravel())
        assert np.array_equal(got_rows, want_rows)
        assert (host[total:] == -1).all()
        one = ctx.detect(*batch[0], leaves_out=out)
        _same(one, want[0])
    with pytest.raises(ValueError):
        ctx.detect_batch(batch, leaves_out=np.zeros((total - 1, 4), np.int32))
    with pytest.raises(ValueError):
        ctx.detect(*batch[0], leaves_out=np.zeros((1, 4), np.int32))


def test_large_leaf_copies_into_pinned_host_memory(ctx, hht):
    # more than 1 MB of leaves: into pinned host memory they are written by a
    # copy kernel through the buffer's device mapping, into device or pageable
    # memory by cudaMemcpyAsync; every route must give the same bytes
    import ctypes
    import torch
    imgs = [synth.plain_1024(index=2), synth.plain_1024(index=3)]
    dev = [(torch.from_numpy(im.points).cuda(), im.W, im.H, im.depth, im.T) for im in imgs]
    ref = [ctx.detect(*x) for x in dev]
    lv = [r.leaves_numpy().copy() for r in ref]
    assert lv[0].nbytes > (1 << 20)
    pinned = torch.full((len(lv[0]) + len(lv[1]) + 3, 4), -1, dtype=torch.int32).pin_memory()
    one = ctx.detect(*dev[0], leaves_out=pinned)
    assert np.array_equal(one.leaves_numpy(), lv[0])
    assert (pinned[len(lv[0]):] == -1).all()
    pinned.fill_(-1)
    both = ctx.detect_batch(dev, leaves_out=pinned)
    for r, want in zip(both, lv):
        assert np.array_equal(r.leaves_numpy(), want)
    assert (pinned[len(lv[0]) + len(lv[1]):] == -1).all()
    pageable = np.full((len(lv[1]), 4), -1, np.int32)
    assert np.array_equal(ctx.detect(*dev[1], leaves_out=pageable).leaves_numpy(), lv[1])
    # second call of the two-call protocol into pinned memory
    r = hht._Result()
    r.leaves = None
    r.leaf_capacity = 0
    lib = hht.load()
    rc = lib.hht_detect(ctx._h, dev[0][0].data_ptr(), imgs[0].n, imgs[0].W, imgs[0].H, imgs[0].depth, imgs[0].T,
                        ctypes.byref(r))
    assert rc == hht.HHT_E_CAPACITY and r.n_leaves == len(lv[0])
    pinned.fill_(-1)
    assert lib.hht_fetch_leaves(ctx._h, 0, pinned.data_ptr(), len(pinned)) == hht.HHT_OK
    assert np.array_equal(pinned[: len(lv[0])].numpy().astype(np.uint32), lv[0])


def test_capacity_two_call_protocol(ctx, hht):
    import ctypes
    img = synth.plain_128()
    want = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    lib = hht.load()
    pts = np.ascontiguousarray(img.points)
    r = hht._Result()
    small = np.zeros((3, 4), np.int32)
    r.leaves = small.ctypes.data
    r.leaf_capacity = 3
    rc = lib.hht_detect(ctx._h, pts.ctypes.data, img.n, img.W, img.H, img.depth, img.T, ctypes.byref(r))
    assert rc == hht.HHT_E_CAPACITY and r.n_leaves == len(want.leaves)
    # the second call of the protocol copies the kept leaves without a new run
    full = np.zeros((int(r.n_leaves), 4), np.int32)
    assert lib.hht_fetch_leaves(ctx._h, 0, full.ctypes.data, 3) == hht.HHT_E_CAPACITY
    assert lib.hht_fetch_leaves(ctx._h, 1, full.ctypes.data, len(full)) == hht.HHT_E_ARG
    assert lib.hht_fetch_leaves(ctx._h, 0, full.ctypes.data, len(full)) == hht.HHT_OK
    assert np.array_equal(full.astype(np.uint32), want.leaves)
    _same(ctx.detect(img.points, img.W, img.H, img.depth, img.T, leaf_capacity=1), want)


def test_deterministic_repeat(ctx, hht):
    # atomics decide the order of voters inside a segment, never a result:
    # repeated runs are byte-identical (ten plain runs, batches, the FHT
    # form, the solution() walk and line extraction)
    img = synth.plain_1024(index=1)
    a = ctx.detect(img.points, img.W, img.H, img.depth, img.T)
    la = a.leaves_numpy().copy()
    lines0 = ctx.lines(0)
    for _ in range(9):
        b = ctx.detect(img.points, img.W, img.H, img.depth, img.T)
        assert np.array_equal(b.leaves_numpy(), la)
        assert np.array_equal(a.stats, b.stats)
    assert np.array_equal(ctx.lines(0), lines0)
    batch = [(im.points, im.W, im.H, im.depth, im.T) for im in synth.batch_256(12)]
    first = [(r.leaves_numpy().copy(), r.stats) for r in ctx.detect_batch(batch)]
    for _ in range(2):
        for (lv, st), r in zip(first, ctx.detect_batch(batch)):
            assert np.array_equal(r.leaves_numpy(), lv) and np.array_equal(r.stats, st)
    f = hht.Context(device=0)
    try:
        f.set_predicate(hht.PREDICATE_FHT)
        f1 = f.detect(img.points, img.W, img.H, img.depth, img.T)
        f2 = f.detect(img.points, img.W, img.H, img.depth, img.T)
        assert np.array_equal(f1.leaves_numpy(), f2.leaves_numpy()) and np.array_equal(f1.stats, f2.stats)
    finally:
        f.close()
    r1, p1 = ctx.detect_removal(img.points, img.W, img.H, img.depth, img.T)
    r2, p2 = ctx.detect_removal(img.points, img.W, img.H, img.depth, img.T)
    assert np.array_equal(r1.leaves_numpy(), r2.leaves_numpy()) and np.array_equal(p1, p2)


# ------------------------------------------------------------------ batches
def test_batch_of_mixed_images_against_oracle(ctx):
    imgs = [synth.random_small(40000 + s, max_side=400, max_n=3000, max_depth=9, max_T=20) for s in range(24)]
    imgs += [synth.plain_128(index=k) for k in range(4)]
    res = ctx.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs])
    for im, r in zip(imgs, res):
        _same(r, oracle.detect(im.points, im.W, im.H, im.depth, im.T))


def test_batch_equals_single_on_mixed_depths(ctx):
    imgs = [synth.batch_image(k) for k in (0, 3, 7, 11)] + [synth.plain_128(index=1)]
    batch = ctx.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs])
    for im, r in zip(imgs, batch):
        one = ctx.detect(im.points, im.W, im.H, im.depth, im.T)
        assert np.array_equal(r.leaves_numpy(), one.leaves_numpy())
        assert np.array_equal(r.stats, one.stats)


def test_batch_256_full_size_sampled(ctx):
    """The 256-image mixed batch at full size, as the benchmark runs it."""
    imgs = synth.batch_256()
    res = ctx.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs])
    rng = np.random.default_rng(1)
    for k in rng.choice(len(imgs), size=24, replace=False):
        im, r = imgs[k], res[k]
        _props(r, im.T, im.depth)
        _sampled_cells(im.points, im.W, im.H, im.depth, r, k=6, seed=int(k))
        shallow = 5
        want = oracle.detect(im.points, im.W, im.H, shallow, im.T)
        # levels 0..shallow-1 do not depend on the depth; at level `shallow` only
        # the tested / votes / tests columns do not
        assert np.array_equal(r.stats[:, :shallow], want.stats[:, :shallow])
        assert np.array_equal(r.stats[:, shallow, [0, 2, 3]], want.stats[:, shallow, [0, 2, 3]])


def test_plain_4096_full_size_sampled(ctx):
    img = synth.plain_4096()
    r = ctx.detect(img.points, img.W, img.H, img.depth, img.T)
    _props(r, img.T, img.depth)
    _sampled_cells(img.points, img.W, img.H, img.depth, r, k=12, seed=4)
    shallow = 6
    want = oracle.detect(img.points, img.W, img.H, shallow, img.T)
    assert np.array_equal(r.stats[:, :shallow], want.stats[:, :shallow])
    assert np.array_equal(r.stats[:, shallow, [0, 2, 3]], want.stats[:, shallow, [0, 2, 3]])


def test_small_budget_splits_the_batch_into_waves(hht):
    """A context whose memory budget holds only part of the batch runs it in
    several waves; every image's result is unchanged."""
    imgs = [synth.batch_image(k) for k in (0, 1, 2, 4, 5, 6)]
    big = hht.Context(device=0)
    ref = [big.detect(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
    big.close()
    small = hht.Context(device=0, mem_budget=1_500_000_000)
    got = small.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs])
    small.close()
    for a, b in zip(ref, got):
        assert np.array_equal(a.leaves_numpy(), b.leaves_numpy())
        assert np.array_equal(a.stats, b.stats)


def test_range_error_in_a_batch_leaves_other_images_intact(ctx, hht):
    """Points outside an image (more than a warp step of them, between valid
    ones) fail that image only; the images around it in the same level
    streams are unchanged."""
    imgs = [synth.plain_128(index=k) for k in range(3)]
    bad = np.concatenate([imgs[1].points[:50], np.full((70, 2), 200, np.int16), imgs[1].points[50:]])
    batch = [(imgs[0].points, 128, 128, 7, 20), (bad, 128, 128, 7, 20), (imgs[2].points, 128, 128, 7, 20)]
    res = ctx.detect_batch(batch, raise_on_error=False)
    assert res[1].status == hht.HHT_E_RANGE
    for k in (0, 2):
        assert res[k].status == hht.HHT_OK
        _same(res[k], oracle.detect(imgs[k].points, 128, 128, 7, 20))


@pytest.mark.parametrize("shape", range(6))
def test_chunks_that_start_and_end_with_dead_records(hht, shape):
    """Points outside their image leave dead records in the level-0 stream.
    Laid out so that whole 128-record chunks are dead and one chunk starts and
    ends with dead records around live ones (both halves, 1024 records each,
    so chunk borders fall on multiples of 128): the image fails with a range
    error and the image after it in the batch is exact."""
    rng = np.random.default_rng(4242)
    n = 1024
    dead = np.zeros(n, bool)
    for lo, hi in ((0, 260), (384, 390), (505, 512), (896, 1024)):
        dead[lo:hi] = True
    assert dead[384] and dead[511] and not dead[390:505].any()
    pts = rng.integers(0, 128, size=(n, 2)).astype(np.int16)
    pts[dead] = (300, 5)
    good = synth.plain_128(index=0)
    c = hht.Context(device=0)
    try:
        c.set_tuning(shape)
        res = c.detect_batch([(pts, 128, 128, 7, 20), (good.points, 128, 128, 7, 20)], raise_on_error=False)
        assert res[0].status == hht.HHT_E_RANGE
        assert res[1].status == hht.HHT_OK
        _same(res[1], oracle.detect(good.points, 128, 128, 7, 20))
    finally:
        c.close()


@pytest.mark.parametrize("shape", range(6))
def test_every_tile_shape_gives_the_same_result(hht, shape):
    """The autotuner may pick any compiled tile shape of the level kernel;
    every shape must give the oracle's result."""
    c = hht.Context(device=0)
    c.set_tuning(shape)
    imgs = [synth.plain_128(index=shape), synth.plain_1024(index=shape % 2),
            synth.random_small(60000 + shape, max_side=300, max_n=3000, max_depth=9, max_T=8)]
    for im in imgs:
        _same(c.detect(im.points, im.W, im.H, im.depth, im.T), oracle.detect(im.points, im.W, im.H, im.depth, im.T))
    res = c.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs])
    for im, r in zip(imgs, res):
        _same(r, oracle.detect(im.points, im.W, im.H, im.depth, im.T))
    c.close()


def test_autotune_picks_a_shape_and_caches_it(hht, tmp_path):
    imgs = [synth.batch_image(k) for k in (0, 1, 2)]
    batch = [(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
    cache = str(tmp_path / "tune.json")
    c = hht.Context(device=0)
    best, times = c.autotune(batch, cache=cache)
    assert 0 <= best < hht.TUNE_SHAPES and len(times) == hht.TUNE_SHAPES and all(t > 0 for t in times)
    assert times[best] == min(times)
    again, t2 = c.autotune(batch, cache=cache)
    assert again == best and t2 is None  # served from the cache
    got = c.detect_batch(batch)
    for im, r in zip(imgs, got):
        _props(r, im.T, im.depth)
    c.close()


def test_graph_form_first_call_is_one_graph_launch_and_later_jobs_replay_it(hht):
    """The default form: a fresh batch runs as one CUDA-graph launch on its
    first call (buffers sized from upper bounds, no earlier run of the job),
    and a later batch of other images with the same deepest level and buffers
    replays the captured graph.  Every result equals the oracle's."""
    c = hht.Context(device=0)
    try:
        c.profile(True)
        first = [synth.plain_128(index=k) for k in range(3)] + [synth.batch_image(0), synth.plain_1024()]
        got = c.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in first])
        for r, im in zip(got, first):
            _same(r, oracle.detect(im.points, im.W, im.H, im.depth, im.T))
        p = c.profile_read()
        assert p["graph_launches"] == 1 and p["graph_captures"] == 1 and p["graph_fallbacks"] == 0, p
        # other images whose bounds are no larger, with the same deepest level
        # (10): the buffers hold them, so the graph is replayed
        big = first[-1]
        later = [(synth.plain_128(index=5).points, 128, 128, 7, 20), (big.points, big.W, big.H, big.depth, 200),
                 (synth.plain_128(index=6).points, 128, 128, 6, 9)]
        for _ in range(2):
            got = c.detect_batch(later)
            for r, x in zip(got, later):
                _same(r, oracle.detect(*x))
        p = c.profile_read()
        assert p["graph_launches"] == 3 and p["graph_captures"] == 1 and p["graph_fallbacks"] == 0, p
    finally:
        c.close()


def test_graph_grids_follow_the_job_and_a_covering_graph_is_replayed(hht):
    """Each level's grids come from the job's own bounds (powers of two), and
    any graph of the same arguments whose grids cover a job's may run it: a
    graph captured for a large job runs a smaller one, while a context that
    saw only the small job captures a second graph for the large one (whose
    buffers are then larger) and replays it for both.  Every result equals
    the oracle's."""
    # the same depth (a graph's arguments include it): 128^2 and 1024^2 at depth 10
    p128 = synth.plain_128(index=2)
    small = (p128.points, 128, 128, 10, 20)
    big = synth.plain_1024()
    large = (big.points, big.W, big.H, big.depth, big.T)
    assert big.depth == 10
    want = {"s": oracle.detect(*small), "l": oracle.detect(*large)}

    def run(c, job, key):
        _same(c.detect(*job, leaves_on_device=False), want[key])
        return c.profile_read()

    c = hht.Context(device=0)
    try:
        c.profile(True)
        p = run(c, large, "l")
        assert p["graph_captures"] == 1 and p["graph_launches"] == 1, p
        p = run(c, small, "s")  # the large job's graph covers it
        assert p["graph_captures"] == 1 and p["graph_launches"] == 2, p
    finally:
        c.close()
    c = hht.Context(device=0)
    try:
        c.profile(True)
        p = run(c, small, "s")
        assert p["graph_captures"] == 1 and p["graph_launches"] == 1, p
        p = run(c, large, "l")  # not covered by the small job's grids
        assert p["graph_captures"] == 2 and p["graph_launches"] == 2, p
        p = run(c, small, "s")  # the large job's buffers and graph now serve both
        p = run(c, large, "l")
        assert p["graph_captures"] == 2 and p["graph_launches"] == 4 and p["graph_fallbacks"] == 0, p
    finally:
        c.close()


def test_graph_and_level_forms_agree(hht):
    """The graph form and the level form (one launch per level, exact sizes)
    give the same leaves and statistics, single images and batches."""
    imgs = [synth.batch_image(k) for k in (2, 9)] + [synth.plain_128(index=7),
                                                    synth.random_small(444, max_side=200, max_n=700,
                                                                       max_depth=8, max_T=4)]
    batch = [(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
    g = hht.Context(device=0)
    lv = hht.Context(device=0)
    try:
        lv.set_batch_mode(hht.BATCH_LEVELS)
        for a, b in zip(g.detect_batch(batch), lv.detect_batch(batch)):
            assert np.array_equal(a.leaves_numpy(), b.leaves_numpy()) and np.array_equal(a.stats, b.stats)
        for x in batch:
            a, b = g.detect(*x), lv.detect(*x)
            assert np.array_equal(a.leaves_numpy(), b.leaves_numpy()) and np.array_equal(a.stats, b.stats)
        assert lv.profile_read()["graph_launches"] == 0
    finally:
        g.close()
        lv.close()


def test_graph_form_overflow_reruns_level_by_level(hht):
    """Host-side injection tells the graph's kernels that the level-1 stream
    holds 10 records: the selection reports the overflow, every later kernel
    of the graph skips its work, and the job is rerun level by level with the
    oracle's result; the next job runs in the graph form again."""
    img = synth.plain_128(index=1)
    want = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    c = hht.Context(device=0)
    try:
        c.profile(True)
        c.inject_fault(hht.FAULT_GRAPH_CAPACITY, 10)
        _same(c.detect(img.points, img.W, img.H, img.depth, img.T), want)
        p = c.profile_read()
        assert p["graph_fallbacks"] == 1 and p["graph_launches"] == 1, p
        _same(c.detect(img.points, img.W, img.H, img.depth, img.T), want)
        p = c.profile_read()
        assert p["graph_fallbacks"] == 1 and p["graph_launches"] == 2, p
    finally:
        c.close()


def test_graph_form_on_a_caller_stream(hht):
    """On a non-default stream the graph is captured on the caller's stream
    and replayed; results stay equal to the oracle's."""
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        c = hht.Context(device=0, stream=s)
        c.profile(True)
        imgs = [synth.plain_128(index=k) for k in range(2)] + [synth.batch_image(1)]
        batch = [(torch.from_numpy(im.points).cuda(), im.W, im.H, im.depth, im.T) for im in imgs]
        want = [oracle.detect(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
        for _ in range(4):
            got = c.detect_batch(batch)
            s.synchronize()
            for r, w in zip(got, want):
                _same(r, w)
        p = c.profile_read()
        assert p["graph_launches"] == 4 and p["graph_captures"] == 1, p
        c.close()


# ------------------------------------------------------------------ one image split by subtrees
@pytest.mark.parametrize("split_level,world", [(1, 2), (2, 3), (3, 4)])
def test_subtree_shards_merge_to_the_whole_detection(ctx, split_level, world):
    # the shards run one after another on this GPU, as separate ranks would;
    # their merge equals the unsharded detection (and, for 128^2, the oracle)
    import torch
    from paper_1007_0547_gb300 import shard
    for img in (synth.plain_128(index=2), synth.plain_1024(index=2)):
        pts = torch.from_numpy(img.points).cuda()
        whole = ctx.detect(pts, img.W, img.H, img.depth, img.T)
        parts = []
        for keep in shard.plan_subtrees(split_level, world):
            r = ctx.detect_subtrees(pts, img.W, img.H, img.depth, img.T, split_level, keep)
            parts.append((r.leaves_numpy(), r.stats))
        lv, st = shard.merge_subtrees(parts, split_level, img.depth)
        assert np.array_equal(lv, whole.leaves_numpy()), (img.name, split_level, world)
        assert np.array_equal(st, whole.stats), (img.name, split_level, world)
        if img.W == 128:
            want = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
            assert np.array_equal(lv, want.leaves) and np.array_equal(st, want.stats)
            one = oracle.detect_subtrees(img.points, img.W, img.H, img.depth, img.T, split_level,
                                         shard.plan_subtrees(split_level, world)[0])
            assert np.array_equal(parts[0][0], one.leaves) and np.array_equal(parts[0][1], one.stats)



# ------------------------------------------------------------------ a caller's allocator
def test_torch_allocator_holds_the_scratch(hht):
    import torch
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated(0)
    c = hht.Context(device=0, allocator="torch")
    try:
        for img in (synth.plain_128(index=1), synth.random_small(4321, max_side=300, max_n=2500, max_depth=9,
                                                                  max_T=10)):
            _same(c.detect(img.points, img.W, img.H, img.depth, img.T),
                  oracle.detect(img.points, img.W, img.H, img.depth, img.T))
        big = synth.plain_1024()
        got = c.detect(big.points, big.W, big.H, big.depth, big.T)
        ref = hht.Context(device=0)
        want = ref.detect(big.points, big.W, big.H, big.depth, big.T)
        ref.close()
        assert np.array_equal(got.leaves_numpy(), want.leaves_numpy())
        assert np.array_equal(got.stats, want.stats)
        # the context's scratch is torch memory while the context lives
        assert torch.cuda.memory_allocated(0) - before > (64 << 20)
    finally:
        c.close()
    del got, want
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated(0) - before < (64 << 20)


def test_batch_calls_that_run_nothing_fetch_nothing(ctx, hht):
    """After a batch of three images, an empty batch returns [] and a batch
    rejected by its argument checks raises HHT_E_ARG (or, without raising,
    reports its image failed with no leaves): neither touches the earlier
    job's leaves or offsets, and the next batch is exact."""
    imgs = [synth.plain_128(index=k) for k in range(3)]
    batch = [(im.points, 128, 128, 7, 20) for im in imgs]
    ctx.detect_batch(batch)
    assert ctx.detect_batch([]) == []
    bad = [(imgs[0].points, 128, 128, 0, 20)]  # depth 0
    with pytest.raises(hht.HhtError) as e:
        ctx.detect_batch(bad)
    assert e.value.code == hht.HHT_E_ARG
    res = ctx.detect_batch(bad, raise_on_error=False)
    assert len(res) == 1 and res[0].status == hht.HHT_E_ARG and res[0].n_leaves == 0
    for r, im in zip(ctx.detect_batch(batch), imgs):
        _same(r, oracle.detect(im.points, 128, 128, 7, 20))
