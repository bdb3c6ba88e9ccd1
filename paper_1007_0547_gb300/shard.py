"""Sharding a batch of images across ranks (one process per GPU).

Images are independent problems, so the hierarchical Hough transform shards
by image with no exchange on the data path: every rank runs its share of the
images through its own context, and the per-image results (leaves and level
statistics, a few KB to MB each) are gathered to rank 0 once at the end.
Shares are balanced by an estimate of each image's work (points x cells per
side, which is proportional to the voter-level count in the dense regime).
"""
from __future__ import annotations

import heapq
from typing import Callable, List, Sequence, Tuple


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
