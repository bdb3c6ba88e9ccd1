"""Serving with continuous batching (hht_submit / hht_progress / hht_poll).

Requests join a running level loop at different steps and share every launch
with the requests already in flight; each result must equal the oracle's and
the same image run alone with hht_detect (exact: results are integers)."""
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


def _alone(hht, imgs):
    ctx = hht.Context(device=0)
    out = [ctx.detect(im.points, im.W, im.H, im.depth, im.T, leaves_on_device=False) for im in imgs]
    ctx.close()
    return out


def _same(a, b):
    assert np.array_equal(a.leaves_numpy(), b.leaves_numpy())
    assert np.array_equal(a.stats, b.stats)


def _mixed_requests():
    imgs = [synth.plain_128(index=k) for k in range(3)]
    imgs += [synth.random_small(900 + s, max_side=300, max_n=2000, max_depth=9, max_T=10) for s in range(6)]
    imgs += [synth.batch_image(k) for k in (0, 1)]
    imgs += [synth.serving_request(k) for k in range(4) if synth.serving_request(k).W <= 1024]
    return imgs


def test_requests_joining_mid_flight_match_alone(hht):
    imgs = _mixed_requests()
    want = _alone(hht, imgs)
    ctx = hht.Context(device=0)
    tickets = {}
    # stagger arrivals: a few requests per step while earlier ones run
    pending = list(range(len(imgs)))
    steps = 0
    results = {}
    while pending or len(results) < len(imgs):
        for _ in range(2):
            if pending:
                k = pending.pop(0)
                im = imgs[k]
                tickets[ctx.submit(im.points, im.W, im.H, im.depth, im.T)] = k
        ctx.progress()
        steps += 1
        for t, k in list(tickets.items()):
            r = ctx.poll(t)
            if r is not None:
                results[k] = r
                del tickets[t]
        assert steps < 500
    for k in range(len(imgs)):
        _same(results[k], want[k])
    ctx.close()


def _oracle_futures(ex, imgs):
    """The oracle's runs of each request, started on the host pool: requests
    with a large n * 2^depth as level-2 subtree shares.  Returns per request
    (split level, futures)."""
    jobs = []
    for im in imgs:
        if im.n * (1 << im.depth) > 500_000_000:
            jobs.append((2, full_oracle.submit_shares(ex, im.points, im.W, im.H, im.depth, im.T, 2)))
        else:
            jobs.append((0, full_oracle.submit_whole(ex, im.points, im.W, im.H, im.depth, im.T)))
    return jobs


def _oracle_result(job, depth):
    split, futs = job
    if split == 0:
        r = futs[0].result()
        return r.leaves, r.stats
    return full_oracle.combine([f.result() for f in futs], split, depth)


def test_serving_stream_against_oracle(hht):
    """The first 40 requests of the serving stream (sides log-uniform in
    64-4096, 1-256 segments, noise 0-3 %, depth ceil(log2 side), T in
    16-256), arriving a few per step while earlier ones run, so that small and
    4096-wide requests share launches: every result equals the oracle's."""
    imgs = synth.serving_requests(40)
    assert max(im.W for im in imgs) > 3500 and min(im.W for im in imgs) < 128
    with full_oracle.pool() as ex:
        # the oracle runs on the host cores while the GPU serves the stream
        # (host threads only: no process is forked after the first GPU call)
        want = _oracle_futures(ex, imgs)
        ctx = hht.Context(device=0)
        try:
            tickets, results, pending, steps = {}, {}, list(range(len(imgs))), 0
            while pending or len(results) < len(imgs):
                for _ in range(3):
                    if pending:
                        k = pending.pop(0)
                        im = imgs[k]
                        tickets[ctx.submit(im.points, im.W, im.H, im.depth, im.T)] = k
                ctx.progress()
                steps += 1
                for t in ctx.done_tickets():
                    results[tickets.pop(t)] = ctx.poll(t)
                assert steps < 5000
        finally:
            ctx.close()
        for k, im in enumerate(imgs):
            lv, st = _oracle_result(want[k], im.depth)
            assert np.array_equal(results[k].stats, st), im.name
            assert np.array_equal(results[k].leaves_numpy(), lv), im.name


def test_small_budget_admits_gradually(hht):
    imgs = [synth.batch_image(k) for k in (2, 4, 5)] + [synth.plain_128(index=4)]
    want = _alone(hht, imgs)
    ctx = hht.Context(device=0, mem_budget=600_000_000)
    tickets = [ctx.submit(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
    got = [None] * len(imgs)
    for _ in range(400):
        left = ctx.progress()
        for i, t in enumerate(tickets):
            if got[i] is None:
                got[i] = ctx.poll(t)
        if all(g is not None for g in got):
            break
    for a, b in zip(got, want):
        _same(a, b)
    ctx.close()


def _bounds(n, W, H, depth, T, horizon=27):
    """Per step k after admission: the request's voter records (lists are
    kept up to level depth - 2; at level l a line votes in at most
    2^l + (W_h - 1) 2^l / (2L) + 2 cells and no more than 4^l) and parent
    regions (levels up to depth - 1; at most 4^l, and its votes / T), both
    halves."""
    L = 1
    while L < max(W, H):
        L *= 2
    stream, regions = [0] * horizon, [0] * horizon
    for l in range(horizon):
        col = 1 << l
        votes = [n * min(col + (Wh - 1) * col // (2 * L) + 2, col * col) for Wh in (W, H)]
        if depth >= 2 and l <= depth - 2:
            stream[l] = 2 * n if l == 0 else sum(votes)
        if l <= depth - 1:
            regions[l] = 2 if l == 0 else sum(min(col * col, v // T) for v in votes)
    return stream, regions


def _need(profiles):
    """Bytes the engine's admission asks for with the given (stream, regions)
    profiles in flight, each shifted by its admission step: the two stream
    buffers at their largest, and the largest step's region buffers."""
    horizon = 40
    st, rg = [0] * horizon, [0] * horizon
    for (stream, regions), shift in profiles:
        for k, (a, b) in enumerate(zip(stream, regions)):
            if k + shift < horizon:
                st[k + shift] += a
                rg[k + shift] += b
    even = max(st[0::2])
    odd = max(st[1::2])
    return 8 * (even + odd) + max(rg) * (16 + 4 * (16 + 16 + 8 + 16))


def test_small_requests_pass_a_blocked_large_one_until_it_has_waited(hht):
    """A large request B that does not fit the budget beside a running one
    (A) is passed over by a small one (C) that does, which finishes first.
    Once B has waited 12 steps, a small request D that arrives is held back
    until B is admitted, although D would fit beside A.  B is admitted at the
    first step where the projection of both walks fits: the admission
    projects each request's voter and region bounds over its coming levels.
    One progress() call is one step; a request of depth d finishes d steps
    after its admission."""
    rng = np.random.default_rng(20261204)
    big = (rng.integers(0, 64, size=(200, 2)).astype(np.int16), 64, 64, 20, 4)  # in flight for 20 steps
    small = (rng.integers(0, 32, size=(10, 2)).astype(np.int16), 32, 32, 3, 1)
    pa = _bounds(200, 64, 64, 20, 4)
    pc = _bounds(10, 32, 32, 3, 1)
    with_c = _need([(pa, 0), (pc, 2)])
    # the admission allows 90 % of the budget: what A and C need, and 64 KiB
    # for the rounding of buffer sizes, so that B fits beside A only late in
    # A's walk (then B's regions no longer add much to A's largest step)
    budget = int((with_c + (64 << 10)) / 0.9) + 1
    t_b = next(t for t in range(1, 40) if _need([(pa, 0), (pa, t)]) <= 0.9 * budget)
    assert 14 <= t_b <= 19, t_b  # B still waits when D comes (step 13: B has waited 12 steps)
    # the engine's buffers are rounded up to 4 KiB, so its sums exceed these
    # by a few KiB at most: B must fit at t_b with room to spare
    assert 0.9 * budget - _need([(pa, 0), (pa, t_b)]) >= 16 << 10
    assert _need([(pa, 0), (pa, t_b), (pc, t_b)]) <= 0.9 * budget  # D fits beside B then

    class _Im:
        def __init__(self, t):
            self.points, self.W, self.H, self.depth, self.T = t

    want = _alone(hht, [_Im(big), _Im(small)])
    ctx = hht.Context(device=0, mem_budget=budget)
    try:
        ta = ctx.submit(*big)
        ctx.progress()                      # step 0: A admitted (the engine was idle)
        tb = ctx.submit(*big)
        ctx.progress()                      # step 1: B does not fit beside A
        tc = ctx.submit(*small)
        done_at, got = {}, {}
        td = None
        for step in range(2, 200):
            if step == 13:                  # B has waited 12 steps: nothing passes it now
                td = ctx.submit(*small)
            ctx.progress()
            for t in ctx.done_tickets():
                done_at[t] = step
                got[t] = ctx.poll(t)
            if len(got) == 4:
                break
        assert len(got) == 4
        assert done_at[tc] == 4             # admitted at step 2 beside A
        assert done_at[ta] == 19
        assert done_at[tb] == t_b + 19      # admitted at step t_b
        assert done_at[td] == t_b + 2       # admitted with B, not at step 13
        for t in (ta, tb):
            _same(got[t], want[0])
        for t in (tc, td):
            _same(got[t], want[1])
    finally:
        ctx.close()


def test_budget_far_below_the_stream_holds(hht):
    """Forty requests of the serving stream submitted at once under a budget
    of a fifth of their summed needs (at least what the largest needs
    alone): admission by projected bounds keeps the engine within it (summed
    peak estimates could not: the two alternating voter buffers each keep
    their own largest size), and every result equals the image run alone."""
    reqs = [synth.serving_request(k) for k in range(40)]
    alone_need = [_need([(_bounds(im.n, im.W, im.H, im.depth, im.T), 0)]) for im in reqs]
    budget = int(max(max(alone_need) / 0.9 * 1.05, sum(alone_need) / 5))
    want = _alone(hht, reqs)
    ctx = hht.Context(device=0, mem_budget=budget)
    try:
        tickets = {ctx.submit(im.points, im.W, im.H, im.depth, im.T): k for k, im in enumerate(reqs)}
        got = {}
        for _ in range(100000):
            ctx.progress()
            for t in ctx.done_tickets():
                got[tickets[t]] = ctx.poll(t)
            if len(got) == len(reqs):
                break
        assert len(got) == len(reqs)
        for k in range(len(reqs)):
            _same(got[k], want[k])
    finally:
        ctx.close()


def test_bad_request_fails_alone(hht):
    good = synth.plain_128(index=1)
    want = _alone(hht, [good])[0]
    ctx = hht.Context(device=0)
    bad_pts = np.array([[5, 3], [40, 2]], np.int16)
    tb = ctx.submit(bad_pts, 32, 32, 5, 1)
    tg = ctx.submit(good.points, good.W, good.H, good.depth, good.T)
    res_g, err = None, None
    for _ in range(50):
        ctx.progress()
        if err is None:
            try:
                if ctx.poll(tb) is not None:
                    err = "no error"
            except hht.HhtError as e:
                err = e.code
        if res_g is None:
            res_g = ctx.poll(tg)
        if res_g is not None and err is not None:
            break
    assert err == hht.HHT_E_RANGE
    _same(res_g, want)
    with pytest.raises(hht.HhtError):
        ctx.poll(tb)  # the ticket was released
    ctx.close()


def test_completion_list_names_each_finished_request_once(hht):
    imgs = _mixed_requests()
    want = _alone(hht, imgs)
    ctx = hht.Context(device=0)
    try:
        tickets = {ctx.submit(im.points, im.W, im.H, im.depth, im.T): k for k, im in enumerate(imgs)}
        seen, got = set(), {}
        for _ in range(100000):
            if len(got) == len(imgs):
                break
            ctx.progress()
            for t in ctx.done_tickets():
                assert t in tickets and t not in seen
                seen.add(t)
                r = ctx.poll(t)
                assert r is not None
                got[tickets[t]] = r
        assert len(got) == len(imgs)
        for k, r in got.items():
            _same(r, want[k])
        assert ctx.done_tickets() == []
    finally:
        ctx.close()


def test_completion_list_stays_bounded_when_only_polled(hht):
    """A client that polls tickets without draining the completion list: the
    list is compacted once polled tickets outnumber the live ones, and a later
    drain names exactly the finished tickets not yet polled, in completion
    order."""
    imgs = [synth.random_small(1700 + s, max_side=64, max_n=60, max_depth=6, max_T=6) for s in range(150)]
    ctx = hht.Context(device=0)
    try:
        tickets = [ctx.submit(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
        for _ in range(100000):
            if ctx.progress() == 0:
                break
        for t in tickets[:-5]:
            assert ctx.poll(t) is not None
        assert sorted(ctx.done_tickets()) == sorted(tickets[-5:])
        assert ctx.done_tickets() == []
        for t in tickets[-5:]:
            assert ctx.poll(t) is not None
    finally:
        ctx.close()
