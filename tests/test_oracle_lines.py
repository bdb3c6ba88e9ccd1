"""Pins of the oracle's leaf -> line step (clusters of touching leaves, one
line per cluster at its peak cell's centre).

- hand-worked clusters (tests/golden/lines_clusters.json);
- cluster membership against networkx connected components (a library
  routine) on random leaf sets, with the peak, cell count and vote total
  recomputed from each component;
- the line of a cell is the cell's centre: strictly inside the cell;
- end to end on exact image lines: the vote-weighted centre of the strongest
  cluster found for points drawn on y = m0 x + b0 (ALPHA) or x = m0 y + b0
  (BETA) lies within a cell of the drawn line's parameters.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lines_clusters.json")


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"][:30])
def test_hand_worked_clusters(case):
    got = oracle.lines(np.array(case["leaves"], dtype=np.uint32).reshape(-1, 4))
    rows = [[int(r["half"]), int(r["i"]), int(r["j"]), int(r["votes"]), int(r["cells"]), int(r["total_votes"]),
             int(r["sum_i2"]), int(r["sum_j2"])] for r in got]
    assert rows == case["lines"]


def test_clusters_against_networkx():
    nx = pytest.importorskip("networkx")
    st = synth.Stream(77)
    for trial in range(20):
        n = int(st.ints(1, 80, 1)[0])
        cells = {}
        while len(cells) < n:
            h, i, j = int(st.ints(0, 1, 1)[0]), int(st.ints(0, 11, 1)[0]), int(st.ints(0, 11, 1)[0])
            cells.setdefault((h, i, j), int(st.ints(1, 9, 1)[0]))
        leaves = np.array([[h, i, j, v] for (h, i, j), v in cells.items()], dtype=np.uint32)
        g = nx.Graph()
        g.add_nodes_from(range(len(leaves)))
        for a in range(len(leaves)):
            for b in range(a + 1, len(leaves)):
                if leaves[a, 0] == leaves[b, 0] and abs(int(leaves[a, 1]) - int(leaves[b, 1])) <= 1 and \
                        abs(int(leaves[a, 2]) - int(leaves[b, 2])) <= 1:
                    g.add_edge(a, b)
        comps = sorted((sorted(c) for c in nx.connected_components(g)), key=lambda c: c[0])
        got = oracle.lines(leaves)
        assert len(got) == len(comps), trial
        for r, comp in zip(got, comps):
            peak = max(comp, key=lambda k: (int(leaves[k, 3]), -k))
            assert (int(r["half"]), int(r["i"]), int(r["j"]), int(r["votes"])) == tuple(int(v) for v in leaves[peak])
            assert int(r["cells"]) == len(comp)
            assert int(r["total_votes"]) == int(leaves[comp, 3].sum())
            v = leaves[comp, 3].astype(np.int64)
            assert int(r["sum_i2"]) == int((v * (2 * leaves[comp, 1].astype(np.int64) + 1)).sum())
            assert int(r["sum_j2"]) == int((v * (2 * leaves[comp, 2].astype(np.int64) + 1)).sum())


def test_line_of_a_cell_is_inside_the_cell():
    for depth, L in ((3, 8), (7, 128), (10, 1024)):
        K = 1 << depth
        for i in (0, 1, K // 2, K - 1):
            for j in (0, 3, K - 1):
                m, b = oracle.line_parameters(0, i, j, depth, L)
                assert Fraction(-K + 2 * i, K) < m < Fraction(-K + 2 * i + 2, K)
                assert Fraction(-2 * L * K + 4 * L * j, K) < b < Fraction(-2 * L * K + 4 * L * (j + 1), K)


@pytest.mark.parametrize("m0,b0,half", [(Fraction(1, 2), 10, 0), (Fraction(-1, 4), 40, 0), (Fraction(1, 4), 3, 1)])
def test_strongest_line_recovers_a_drawn_line(m0, b0, half):
    W = H = 64
    pts = []
    for u in range(64):
        v = m0 * u + b0
        if v.denominator == 1 and 0 <= v < 64:
            pts.append((u, int(v)) if half == 0 else (int(v), u))
    pts = np.array(pts, dtype=np.int16)
    depth, T = 6, len(pts) - 2
    res = oracle.detect(pts, W, H, depth, T)
    lines = oracle.lines(res.leaves)
    lines = lines[lines["half"] == half]
    best = lines[np.argmax(lines["total_votes"])]
    K = 1 << depth
    # the cluster's vote-weighted centre lies within a cell of the drawn line
    m, b = oracle.centroid_parameters(best, depth, 64)
    assert abs(m - m0) <= Fraction(2, K) and abs(b - b0) <= Fraction(4 * 64, K)
    # and its peak cell touches the drawn line's cluster: within the cluster's extent
    pm, pb = oracle.line_parameters(half, int(best["i"]), int(best["j"]), depth, 64)
    assert abs(pm - m0) <= Fraction(2 * int(best["cells"]), K)
