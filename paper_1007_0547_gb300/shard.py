"""Sharding across ranks (one process per GPU).

Across images: images are independent problems, so the hierarchical Hough
transform shards by image with no exchange on the data path: every rank runs
its share of the images through its own context, and the per-image results
(leaves and level statistics, a few KB to MB each) are gathered to rank 0
once at the end.  Shares are balanced by an estimate of each image's work
(points x cells per side, which is proportional to the voter-level count in
the dense regime).

Within one image: below a split level k the 2 * 4^k subtrees of the two
halves are independent given the (replicated) points, because a region's
votes come only from the lines that cross it.  Every rank runs levels 0..k
in full and continues only below its own level-k regions
(hht_detect_subtrees); leaves are then merged in depth-first order and the
level statistics combined (levels below k are the same on every rank; at
level k the pass counts add up; below k every count adds up).
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Sequence, Tuple

import numpy as np


def image_work(n: int, depth: int) -> float:
    """Work estimate of one image: every point's line crosses about 1.25 * 2^l
    cells at level l, so the voter-levels grow as n * 2^depth."""
    return float(max(n, 1)) * float(2 ** depth)


def plan_shards(images: Sequence[Tuple], world: int) -> List[List[int]]:
    """Partition image indices into `world` shares of near-equal estimated work
    (longest processing time first; each share keeps the original order).
    images: (points, W, H, depth, T) tuples."""
    if world < 1:
        raise ValueError("world must be >= 1")
    work = []
    for k, im in enumerate(images):
        pts = im[0]
        n = int(pts.shape[0]) if hasattr(pts, "shape") else len(pts)
        work.append((image_work(n, int(im[3])), k))
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    shares: List[List[int]] = [[] for _ in range(world)]
    for w, k in sorted(work, key=lambda t: (-t[0], t[1])):
        load, r = heapq.heappop(heap)
        shares[r].append(k)
        heapq.heappush(heap, (load + w, r))
    return [sorted(s) for s in shares]


def run_sharded(images: Sequence[Tuple], detect_batch: Callable[[List[Tuple]], list], rank: int, world: int,
                gather: Callable[[object], list]) -> list:
    """Run this rank's share with `detect_batch` and gather every share's
    results; rank 0 gets the results of all images in the original order
    (other ranks get None).  `gather(obj)` must return the list of all ranks'
    objects on rank 0 (e.g. torch.distributed.gather_object) and anything on
    the other ranks."""
    shares = plan_shards(images, world)
    mine = shares[rank]
    local = detect_batch([images[k] for k in mine]) if mine else []
    collected = gather((mine, local))
    if rank != 0:
        return None
    out = [None] * len(images)
    for idx, res in collected:
        for k, r in zip(idx, res):
            out[k] = r
    return out


def dfs_key(i, j, depth: int):
    """Position of cell (i, j) of a depth-`depth` grid in the depth-first
    order of the hierarchy (children NE, NW, SW, SE at every level); works on
    integers and on integer numpy arrays."""
    key = np.zeros(np.shape(i), dtype=np.int64)
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    for lvl in range(depth - 1, -1, -1):
        east, north = (i >> lvl) & 1, (j >> lvl) & 1
        q = np.where(north == 1, np.where(east == 1, 0, 1), np.where(east == 1, 3, 2))
        key = key * 4 + q
    return key


def plan_subtrees(split_level: int, world: int) -> List[np.ndarray]:
    """Keep masks (uint8 [2 * 4^k], entry half * 4^k + a * 2^k + b) that deal
    the level-k regions (a, b) of both halves round-robin to `world` ranks in
    depth-first order, so that neighbouring (similarly loaded) regions go to
    different ranks."""
    if world < 1 or split_level < 1:
        raise ValueError("world >= 1 and split_level >= 1 needed")
    side = 1 << split_level
    a, b = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    a, b = a.ravel(), b.ravel()
    order = np.argsort(dfs_key(a, b, split_level), kind="stable")
    masks = [np.zeros(2 * side * side, dtype=np.uint8) for _ in range(world)]
    pos = 0
    for half in (0, 1):
        for idx in order:
            masks[pos % world][half * side * side + a[idx] * side + b[idx]] = 1
            pos += 1
    return masks


def merge_subtrees(parts: Sequence[Tuple[np.ndarray, np.ndarray]], split_level: int, depth: int):
    """Combine the (leaves [k, 4], stats [2, depth + 1, 4]) of the ranks of a
    detection split by level-`split_level` subtrees into the whole
    detection's: leaves in depth-first order (half 0 first), statistics with
    levels < k from rank 0, level k's tested / votes / tests from rank 0 and
    its passed counts summed, levels > k summed."""
    lv = np.concatenate([np.asarray(p[0]).reshape(-1, 4) for p in parts]) if parts else np.zeros((0, 4))
    if len(lv):
        key = (lv[:, 0].astype(np.int64) << 50) | dfs_key(lv[:, 1], lv[:, 2], depth)
        lv = lv[np.argsort(key, kind="stable")]
    st = np.array(parts[0][1], dtype=np.uint64, copy=True)
    k = split_level
    for p in parts[1:]:
        other = np.asarray(p[1], dtype=np.uint64)
        st[:, k, 1] += other[:, k, 1]
        st[:, k + 1:, :] += other[:, k + 1:, :]
    return lv, st


def run_subtree_sharded(image: Tuple, detect_subtrees: Callable, split_level: int, rank: int, world: int,
                        gather: Callable[[object], list]):
    """This rank's subtrees of one image with `detect_subtrees(image,
    split_level, keep) -> (leaves, stats)`, gathered and merged on rank 0
    (None on the other ranks)."""
    keep = plan_subtrees(split_level, world)[rank]
    part = detect_subtrees(image, split_level, keep)
    collected = gather(part)
    if rank != 0:
        return None
    return merge_subtrees(collected, split_level, int(image[3]))
