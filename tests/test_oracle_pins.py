"""Pins of the CPU oracle against things other than itself (CPU only).

- hand-worked codes, leaves and statistics (tests/golden/, Sections 2-3),
- a concurrency vertex where the four surrounding cells' counts follow from
  the tie rule and the corner order alone (tests/golden/concurrent_vertex.json),
- brute force from the paper's definition with exact rationals (tests/pins.py),
- a closed-form column-interval accumulator at full size (tests/pins.py),
- invariants: code alphabet, monotone voter sets, transpose symmetry,
  T > n, single-line cases, statistics identities,
- the FHT circle test: exact voters are a subset of circle voters.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from tests import pins

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _as_list(leaves):
    """Leaves as a list sorted by (half, i, j) (the pins produce that order)."""
    return sorted(tuple(int(v) for v in r) for r in np.asarray(leaves).reshape(-1, 4))



# ----------------------------------------------------------------- hand-worked examples
def test_hand_codes_bit_order_and_tie_rule():
    g = _load("hand_2x2.json")
    L = oracle.frame_side(2, 2)
    assert L == 2
    for pk, cells in g["codes"].items():
        x, y = map(int, pk.split(","))
        for ck, code in cells.items():
            i, j = map(int, ck.split(","))
            assert format(oracle.getcode(x, y, i, j, 1, L, 1), "04b") == code, (pk, ck)


@pytest.mark.parametrize("case", range(3))
def test_hand_leaves_and_stats(case):
    c = _load("hand_2x2.json")["cases"][case]
    r = oracle.detect(np.array(c["points"]), c["W"], c["H"], c["depth"], c["T"])
    assert _as_list(r.leaves) == [tuple(v) for v in c["leaves"]]
    assert r.stats.tolist() == c["stats"]


@pytest.mark.parametrize("case", range(2))
def test_concurrency_vertex(case):
    c = _load("concurrent_vertex.json")["cases"][case]
    pts = np.array(c["points"])
    n = len(pts)
    r = oracle.detect(pts, c["W"], c["H"], c["depth"], 1)
    got = {(int(i), int(j)): int(v) for h, i, j, v in r.leaves if h == 0}
    for role, (i, j, want) in c["half0_cells"].items():
        assert got.get((i, j), 0) == want, role
    # threshold reading: a region passes when votes >= T (so T = n keeps the two
    # full cells, T = n + 1 keeps nothing of half 0 at this vertex)
    full = {(c["half0_cells"]["ne_corner_at_v"][0], c["half0_cells"]["ne_corner_at_v"][1]),
            (c["half0_cells"]["nw_corner_at_v"][0], c["half0_cells"]["nw_corner_at_v"][1])}
    r_eq = oracle.detect(pts, c["W"], c["H"], c["depth"], n)
    kept = {(int(i), int(j)) for h, i, j, v in r_eq.leaves if h == 0}
    assert full <= kept
    assert all(int(v) == n for h, i, j, v in r_eq.leaves)
    r_gt = oracle.detect(pts, c["W"], c["H"], c["depth"], n + 1)
    assert len(r_gt.leaves) == 0


def test_concurrency_vertex_at_the_largest_frame():
    """The concurrency pin at the largest frame and depth (L = 2^15, K = 2^24),
    where the exact corner values reach 2^41.  Points with even x on the image
    line y = x/2 + 100 give parameter-space lines that all pass through
    (m, b) = (1/2, 100), which is the grid vertex (i, j) = (3 * 2^22,
    65636 * 128) at depth 24.  Around it the cells whose NE and NW corners are
    the vertex get every line, the one whose SE corner it is gets the lines
    with x > 0, and the one whose SW corner it is gets none."""
    W = H = 32767
    D, K, L = 24, 1 << 24, 1 << 15
    xs = [0, 2, 4, 6, 8, 10, 12, 14, 16, 18, 20, 22, 30000, 32766]
    pts = np.array([[x, x // 2 + 100] for x in xs], np.int16)
    n, pos = len(xs), sum(1 for x in xs if x > 0)
    i, j = 3 << 22, 65636 * 128
    assert Fraction(-1) + Fraction(2 * i, K) == Fraction(1, 2)
    assert Fraction(-2 * L) + Fraction(4 * L * j, K) == 100
    r = oracle.detect(pts, W, H, D, pos)
    got = {(int(a), int(b)): int(v) for h, a, b, v in r.leaves if h == 0}
    assert got.get((i - 1, j - 1)) == n      # NE corner at the vertex
    assert got.get((i, j - 1)) == n          # NW corner
    assert got.get((i - 1, j)) == pos        # SE corner: the lines with x > 0
    assert (i, j) not in got                 # SW corner: no line
    assert len(oracle.detect(pts, W, H, D, n + 1).leaves) == 0


# ----------------------------------------------------------------- brute force
BRUTE_SEEDS = list(range(120))


@pytest.mark.parametrize("seed", BRUTE_SEEDS)
def test_brute_force_small(seed):
    img = synth.random_small(1000 + seed, max_side=16, max_n=40, max_depth=4, max_T=6)
    want_leaves, want_stats = pins.brute_force(img.points, img.W, img.H, img.depth, img.T)
    r = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    assert _as_list(r.leaves) == want_leaves
    assert r.stats.astype(np.int64).tolist() == want_stats.tolist()


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_depth5(seed):
    img = synth.random_small(5000 + seed, max_side=12, max_n=12, max_depth=5, max_T=3)
    img.depth = 5
    want_leaves, want_stats = pins.brute_force(img.points, img.W, img.H, img.depth, img.T)
    r = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    assert _as_list(r.leaves) == want_leaves
    assert r.stats.astype(np.int64).tolist() == want_stats.tolist()


def test_brute_force_non_square_and_odd_sides():
    st = synth.Stream(77)
    for W, H, D in [(3, 7, 3), (16, 5, 4), (9, 9, 3), (1, 1, 2), (1, 13, 3)]:
        n = 20
        pts = np.stack([st.ints(0, W - 1, n), st.ints(0, H - 1, n)], axis=1)
        for T in (1, 3):
            want_leaves, want_stats = pins.brute_force(pts, W, H, D, T)
            r = oracle.detect(pts, W, H, D, T)
            assert _as_list(r.leaves) == want_leaves, (W, H, D, T)
            assert r.stats.astype(np.int64).tolist() == want_stats.tolist(), (W, H, D, T)


# ----------------------------------------------------------------- closed form at scale
def test_closed_form_plain_128():
    img = synth.plain_128()
    want_leaves, want_stats = pins.closed_form(img.points, img.W, img.H, img.depth, img.T)
    r = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    assert _as_list(r.leaves) == want_leaves
    assert r.stats.astype(np.int64).tolist() == want_stats.tolist()


@pytest.mark.parametrize("k", [3, 17])
def test_closed_form_batch_images_small_sides(k):
    # batch image k, cut to its 256x256 corner so the oracle stays fast
    img = synth.batch_image(k)
    pts = img.points[(img.points[:, 0] < 256) & (img.points[:, 1] < 256)]
    want_leaves, want_stats = pins.closed_form(pts, 256, 256, 8, 16)
    r = oracle.detect(pts, 256, 256, 8, 16)
    assert _as_list(r.leaves) == want_leaves
    assert r.stats.astype(np.int64).tolist() == want_stats.tolist()


@pytest.mark.slow
def test_closed_form_plain_1024():
    img = synth.plain_1024()
    want_leaves, want_stats = pins.closed_form(img.points, img.W, img.H, img.depth, img.T)
    r = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    assert _as_list(r.leaves) == want_leaves
    assert r.stats.astype(np.int64).tolist() == want_stats.tolist()


# ----------------------------------------------------------------- invariants
def test_code_alphabet():
    """For x >= 0 the sign function is monotone in m and b, so only codes
    0000, 1111, 0010, 0011, 0110, 0111 can occur."""
    st = synth.Stream(5)
    allowed = {0, 15, 2, 3, 6, 7}
    for _ in range(2000):
        D = int(st.ints(1, 12, 1)[0])
        W = int(st.ints(1, 4096, 1)[0])
        L = oracle.frame_side(W, W)
        x, y = (int(v) for v in st.ints(0, W - 1, 2))
        lvl = int(st.ints(0, D, 1)[0])
        S = (1 << D) >> lvl
        a, b = (int(v) for v in st.ints(0, (1 << lvl) - 1, 2))
        assert oracle.getcode(x, y, a * S, b * S, S, L, D) in allowed


def test_leaves_come_in_depth_first_order():
    for k in range(3):
        img = synth.plain_128(index=k)
        r = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
        keys = [(int(h), pins.dfs_key(int(i), int(j), img.depth)) for h, i, j, v in r.leaves]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_transpose_symmetry():
    img = synth.plain_128(index=2)
    r = oracle.detect(img.points, img.W, img.H, img.depth, img.T)
    rt = oracle.detect(img.points[:, ::-1], img.H, img.W, img.depth, img.T)
    swapped = rt.leaves.copy()
    swapped[:, 0] = 1 - swapped[:, 0]
    assert _as_list(r.leaves) == _as_list(swapped)
    assert np.array_equal(r.stats[0], rt.stats[1]) and np.array_equal(r.stats[1], rt.stats[0])


def test_threshold_above_n_gives_nothing():
    img = synth.plain_128(index=1)
    r = oracle.detect(img.points, img.W, img.H, img.depth, img.n + 1)
    assert len(r.leaves) == 0
    assert (r.stats[:, 1:, oracle.STAT_PASSED] == 0).all()
    assert (r.stats[:, 1, oracle.STAT_TESTED] == 4).all()


def test_empty_input():
    r = oracle.detect(np.zeros((0, 2), np.int16), 64, 32, 5, 1)
    assert len(r.leaves) == 0
    assert r.stats[:, 0].tolist() == [[1, 1, 0, 0], [1, 1, 0, 0]]
    assert (r.stats[:, 1] == [4, 0, 0, 0]).all()
    assert (r.stats[:, 2:] == 0).all()


def test_single_line_leaves_are_its_crossed_cells():
    st = synth.Stream(9)
    for _ in range(20):
        W = int(st.ints(1, 300, 1)[0])
        H = int(st.ints(1, 300, 1)[0])
        D = int(st.ints(1, 9, 1)[0])
        pt = np.array([[int(st.ints(0, W - 1, 1)[0]), int(st.ints(0, H - 1, 1)[0])]])
        r = oracle.detect(pt, W, H, D, 1)
        for half in (0, 1):
            c = pins.column_counts(pt, W, H, D, D, half)
            want = sorted((half, int(a), int(b), 1) for a, b in zip(*np.nonzero(c)))
            assert [t for t in _as_list(r.leaves) if t[0] == half] == want


@pytest.mark.parametrize("k", range(4))
def test_stats_identities(k):
    img = synth.plain_128(index=k)
    r = oracle.detect(img.points, img.W, img.H, img.depth, img.T, dump_regions=True)
    s = r.stats
    for h in (0, 1):
        assert s[h, 0].tolist() == [1, 1, img.n, img.n]
        for l in range(1, img.depth + 1):
            assert s[h, l, 0] == 4 * s[h, l - 1, 1]
            assert s[h, l, 2] >= img.T * s[h, l, 1]
        assert s[h, img.depth, 1] == int((r.leaves[:, 0] == h).sum())
    # passed-region votes at level l-1 (x4) are the code evaluations at level l
    reg = r.regions
    for h in (0, 1):
        for l in range(1, img.depth + 1):
            par = reg[(reg[:, 0] == h) & (reg[:, 1] == l - 1)]
            passed_votes = par[(par[:, 5] >= img.T) | (l - 1 == 0), 5].sum()
            assert s[h, l, 3] == 4 * passed_votes


def test_voter_sets_are_monotone_down_the_tree():
    """A child's count never exceeds its parent's (child voters are parent voters)."""
    img = synth.plain_128(index=3)
    r = oracle.detect(img.points, img.W, img.H, img.depth, 1, dump_regions=True)
    reg = r.regions
    key = {(int(h), int(l), int(i0), int(j0)): int(v) for h, l, i0, j0, sz, v in reg}
    for h, l, i0, j0, sz, v in reg:
        if l == 0:
            continue
        psz = 2 * int(sz)
        parent = (int(h), int(l) - 1, (int(i0) // psz) * psz, (int(j0) // psz) * psz)
        assert v <= key[parent]


def test_range_and_argument_errors():
    with pytest.raises(ValueError):
        oracle.detect(np.array([[5, 0]]), 5, 5, 3, 1)
    with pytest.raises(ValueError):
        oracle.detect(np.array([[0, -1]]), 5, 5, 3, 1)
    with pytest.raises(ValueError):
        oracle.detect(np.array([[0, 0]]), 5, 5, 0, 1)
    with pytest.raises(ValueError):
        oracle.detect(np.array([[0, 0]]), 5, 5, 3, 0)


# ----------------------------------------------------------------- FHT circle test
def _region_map(res):
    return {(int(h), int(l), int(i0), int(j0)): int(v) for h, l, i0, j0, sz, v in res.regions}


@pytest.mark.parametrize("k", range(3))
def test_exact_votes_subset_of_fht(k):
    img = synth.plain_128(index=k)
    ex = oracle.detect(img.points, img.W, img.H, img.depth, img.T, dump_regions=True)
    fh = oracle.detect(img.points, img.W, img.H, img.depth, img.T, mode="fht", dump_regions=True)
    em, fm = _region_map(ex), _region_map(fh)
    assert set(em) <= set(fm)                    # every exactly tested region is FHT-tested
    for key, v in em.items():
        assert v <= fm[key]                      # exact voters are circle voters
    assert fh.total_votes() >= ex.total_votes()  # C_v >= 1


def test_fht_predicate_contains_exact_predicate():
    st = synth.Stream(11)
    for _ in range(3000):
        D = int(st.ints(1, 10, 1)[0])
        W = int(st.ints(1, 2048, 1)[0])
        L = oracle.frame_side(W, W)
        x, y = (int(v) for v in st.ints(0, W - 1, 2))
        lvl = int(st.ints(0, D, 1)[0])
        S = (1 << D) >> lvl
        a, b = (int(v) for v in st.ints(0, (1 << lvl) - 1, 2))
        code = oracle.getcode(x, y, a * S, b * S, S, L, D)
        if code not in (0, 15):
            assert oracle.fht_votes(x, y, a * S, b * S, S, L, D)


def test_fht_brute_force_tiny():
    """FHT hierarchy == direct circle count over all points: the circle test
    written out on the rational region centre, compared squared and exactly."""
    from fractions import Fraction
    st = synth.Stream(21)
    for trial in range(8):
        W = H = 8
        D, T = 3, 2
        n = 10
        pts = np.stack([st.ints(0, W - 1, n), st.ints(0, H - 1, n)], axis=1)
        fh = oracle.detect(pts, W, H, D, T, mode="fht", dump_regions=True)
        L, K = 8, 8
        for (h, l, i0, j0), v in _region_map(fh).items():
            S = K >> l
            cnt = 0
            for x, y in pins.half_points(pts, h):
                # distance in cell units from centre to the line 4L j + 2x i - 2LK - Kx - Ky = 0
                ci, cj = Fraction(2 * i0 + S, 2), Fraction(2 * j0 + S, 2)
                g = 4 * L * cj + 2 * int(x) * ci - 2 * L * K - K * int(x) - K * int(y)
                # compare squared distance with squared radius S^2 / 2 exactly
                if g * g * 2 <= S * S * (4 * int(x) ** 2 + 16 * L * L):
                    cnt += 1
            assert cnt == v, (trial, h, l, i0, j0)


def test_count_region_matches_hierarchy_and_closed_form():
    img = synth.plain_128(index=1)
    r = oracle.detect(img.points, img.W, img.H, img.depth, 1)
    for h, i, j, v in r.leaves[:: max(1, len(r.leaves) // 40)]:
        assert oracle.count_region(img.points, img.W, img.H, img.depth, int(h), int(i), int(j), 1) == int(v)
    for half in (0, 1):
        c = pins.column_counts(img.points, img.W, img.H, img.depth, 4, half)
        S = 1 << (img.depth - 4)
        for a in range(0, 16, 3):
            for b in range(0, 16, 5):
                assert oracle.count_region(img.points, img.W, img.H, img.depth, half, a * S, b * S, S) == c[a, b]
