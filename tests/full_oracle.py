"""The oracle at full size, on all host cores (test infrastructure).

The C oracle releases the GIL inside its ctypes calls, so a thread pool runs
one detection per core.  An image too large for one thread in a test's time is
split into level-k subtree shares with the oracle's own subtree mode: share r
keeps one level-k region and tests, counts and leaves every other region of
that level unsplit.  The whole detection then follows from the definitions,
restated here without any of the library's code:
  - the leaves are the shares' leaves, shares taken in the depth-first order of
    their level-k regions (half 0 first, children NE, NW, SW, SE), since every
    leaf lies below exactly one level-k region;
  - levels below k: every share holds the whole detection's statistics;
  - level k: tested, votes and code evaluations likewise; a share counts a
    region as passed only when it keeps it, so the passed column is the sum;
  - levels below that: each region lies in exactly one share, so every column
    is the sum over the shares.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from typing import List, Tuple

import numpy as np

import oracle
from tests import pins


def pool(threads: int = 0) -> ThreadPoolExecutor:
    return ThreadPoolExecutor(max_workers=threads or max(1, os.cpu_count() or 1))


def share_masks(split_level: int) -> List[np.ndarray]:
    """One keep mask per level-k region of both halves, in depth-first order."""
    side = 1 << split_level
    regions = np.array([(h, a, b, 0) for h in (0, 1) for a in range(side) for b in range(side)], np.int64)
    order = np.argsort(pins.dfs_keys(regions, split_level), kind="stable")
    masks = []
    for r in order:
        h, a, b = (int(v) for v in regions[r, :3])
        m = np.zeros(2 * side * side, np.uint8)
        m[h * side * side + a * side + b] = 1
        masks.append(m)
    return masks


def submit_whole(ex: ThreadPoolExecutor, points, W: int, H: int, depth: int, T: int):
    return [ex.submit(oracle.detect, points, W, H, depth, T)]


def submit_shares(ex: ThreadPoolExecutor, points, W: int, H: int, depth: int, T: int, split_level: int):
    return [ex.submit(oracle.detect_subtrees, points, W, H, depth, T, split_level, m)
            for m in share_masks(split_level)]


def combine(results, split_level: int, depth: int) -> Tuple[np.ndarray, np.ndarray]:
    """(leaves, stats) of the whole detection from its shares (module docstring)."""
    k = split_level
    leaves = np.concatenate([r.leaves for r in results]).reshape(-1, 4) if results else np.zeros((0, 4), np.uint32)
    st = np.zeros((2, depth + 1, 4), np.uint64)
    first = results[0].stats
    for r in results[1:]:
        assert np.array_equal(r.stats[:, :k], first[:, :k]), "levels above the split differ between shares"
        assert np.array_equal(r.stats[:, k, [0, 2, 3]], first[:, k, [0, 2, 3]]), "split level differs"
    st[:, :k] = first[:, :k]
    st[:, k, [0, 2, 3]] = first[:, k, [0, 2, 3]]
    st[:, k, 1] = sum(r.stats[:, k, 1] for r in results)
    for r in results:
        st[:, k + 1:] += r.stats[:, k + 1:]
    return np.ascontiguousarray(leaves), st


def detect(points, W: int, H: int, depth: int, T: int, split_level: int = 0, ex=None):
    """(leaves, stats) of the oracle, whole (split_level 0) or by subtree shares."""
    own = ex is None
    ex = ex or pool()
    try:
        if split_level == 0:
            r = submit_whole(ex, points, W, H, depth, T)[0].result()
            return r.leaves, r.stats
        futs = submit_shares(ex, points, W, H, depth, T, split_level)
        return combine([f.result() for f in futs], split_level, depth)
    finally:
        if own:
            ex.shutdown()
