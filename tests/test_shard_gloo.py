"""Multi-rank sharding on CPU with the gloo backend (world sizes 2 and 3).

Across images: each rank detects its share of the images (the CPU oracle
stands in for the GPU here) and rank 0 gathers the results; the merged list
must equal the unsharded run image by image.  Within one image: each rank
runs its level-k subtrees (the oracle's subtree mode), rank 0 merges, and the
merged leaves and statistics must equal the unsharded detection.  The
benchmark's reference arm under torchrun prints one line, from rank 0."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _oracle_batch(batch):
    import oracle
    return [oracle.detect(p, W, H, D, T) for (p, W, H, D, T) in batch]


def _worker(rank, world, port, images, out_path):
    import pickle

    import torch.distributed as dist

    from paper_1007_0547_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def gather(obj):
        objs = [None] * world if rank == 0 else None
        dist.gather_object(obj, objs, dst=0)
        return objs

    merged = shard.run_sharded(images, _oracle_batch, rank, world, gather)
    if rank == 0:
        with open(out_path, "wb") as f:
            pickle.dump([(r.leaves, r.stats) for r in merged], f)
    dist.barrier()
    dist.destroy_process_group()


def test_plan_shards_balances_and_covers():
    from paper_1007_0547_gb300 import shard
    imgs = [synth.batch_image(k) for k in range(12)]
    batch = [(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
    for world in (1, 2, 3, 5):
        shares = shard.plan_shards(batch, world)
        assert sorted(k for s in shares for k in s) == list(range(len(batch)))
        loads = [sum(shard.image_work(len(batch[k][0]), batch[k][3]) for k in s) for s in shares]
        biggest = max(shard.image_work(len(b[0]), b[3]) for b in batch)
        assert max(loads) - min(loads) <= biggest  # greedy bound


def test_two_gloo_ranks_merge_equals_unsharded(tmp_path):
    import pickle

    import torch.multiprocessing as mp
    imgs = [synth.plain_128(index=k) for k in range(4)] + \
        [synth.random_small(70 + s, max_side=200, max_n=800, max_depth=7, max_T=6) for s in range(3)]
    batch = [(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
    out = str(tmp_path / "merged.pkl")
    mp.start_processes(_worker, args=(2, _free_port(), batch, out), nprocs=2, join=True, start_method="spawn")
    with open(out, "rb") as f:
        merged = pickle.load(f)
    want = _oracle_batch(batch)
    assert len(merged) == len(want)
    for (lv, st), w in zip(merged, want):
        assert np.array_equal(lv, w.leaves)
        assert np.array_equal(st, w.stats)


def _subtree_worker(rank, world, port, image, split_level, out_path):
    import pickle

    import torch.distributed as dist

    import oracle
    from paper_1007_0547_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def gather(obj):
        objs = [None] * world if rank == 0 else None
        dist.gather_object(obj, objs, dst=0)
        return objs

    def detect_subtrees(im, k, keep):
        r = oracle.detect_subtrees(im[0], im[1], im[2], im[3], im[4], k, keep)
        return r.leaves, r.stats

    merged = shard.run_subtree_sharded(image, detect_subtrees, split_level, rank, world, gather)
    if rank == 0:
        with open(out_path, "wb") as f:
            pickle.dump(merged, f)
    dist.barrier()
    dist.destroy_process_group()


def test_plan_subtrees_covers_every_region_once():
    from paper_1007_0547_gb300 import shard
    for k in (1, 2, 3):
        for world in (1, 2, 3, 7):
            masks = shard.plan_subtrees(k, world)
            total = np.sum(np.stack(masks).astype(np.int64), axis=0)
            assert np.all(total == 1)
            sizes = [int(m.sum()) for m in masks]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("split_level", [1, 2, 3])
def test_two_gloo_ranks_split_one_image_by_subtrees(tmp_path, split_level):
    import pickle

    import oracle
    import torch.multiprocessing as mp
    img = synth.plain_128(index=3)
    image = (img.points, img.W, img.H, img.depth, img.T)
    out = str(tmp_path / "merged.pkl")
    mp.start_processes(_subtree_worker, args=(2, _free_port(), image, split_level, out), nprocs=2, join=True,
                       start_method="spawn")
    with open(out, "rb") as f:
        lv, st = pickle.load(f)
    want = oracle.detect(*image)
    assert np.array_equal(lv, want.leaves)
    assert np.array_equal(st, want.stats)


def test_three_gloo_ranks_with_an_empty_share(tmp_path):
    """More ranks than images: one rank's share is empty, it still takes part
    in the gather, and the merged list is the unsharded one."""
    import pickle

    import torch.multiprocessing as mp
    imgs = [synth.random_small(90 + s, max_side=120, max_n=400, max_depth=6, max_T=5) for s in range(2)]
    batch = [(im.points, im.W, im.H, im.depth, im.T) for im in imgs]
    from paper_1007_0547_gb300 import shard
    assert sum(1 for s in shard.plan_shards(batch, 3) if not s) == 1
    out = str(tmp_path / "merged.pkl")
    mp.start_processes(_worker, args=(3, _free_port(), batch, out), nprocs=3, join=True, start_method="spawn")
    with open(out, "rb") as f:
        merged = pickle.load(f)
    want = _oracle_batch(batch)
    assert len(merged) == len(want)
    for (lv, st), w in zip(merged, want):
        assert np.array_equal(lv, w.leaves)
        assert np.array_equal(st, w.stats)


def test_three_gloo_ranks_split_one_image_by_subtrees(tmp_path):
    import pickle

    import oracle
    import torch.multiprocessing as mp
    img = synth.plain_128(index=1)
    image = (img.points, img.W, img.H, img.depth, img.T)
    out = str(tmp_path / "merged.pkl")
    mp.start_processes(_subtree_worker, args=(3, _free_port(), image, 2, out), nprocs=3, join=True,
                       start_method="spawn")
    with open(out, "rb") as f:
        lv, st = pickle.load(f)
    want = oracle.detect(*image)
    assert np.array_equal(lv, want.leaves)
    assert np.array_equal(st, want.stats)


def test_bench_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    repo = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    run = subprocess.run(cmd, cwd=repo, capture_output=True, text=True, timeout=600)
    assert run.returncode == 0, run.stderr[-3000:]
    lines = [ln for ln in run.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, run.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["steps"] == 1
    assert rec["value"] > 0 and rec["e2e"]["value"] == rec["value"]
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1


@pytest.mark.parametrize("split_level", [1, 2, 3])
def test_one_shard_keeps_exactly_the_leaves_below_its_regions(split_level):
    """The keep mask's layout (entry half * 4^k + a * 2^k + b for the level-k
    region (a, b)): a shard's leaves are the unsharded leaves whose level-k
    ancestor, (i >> (D - k), j >> (D - k)), it keeps; its statistics below k
    are those of the unsharded run and at level k it passes only kept regions."""
    import oracle
    img = synth.plain_128(index=2)
    D, k = img.depth, split_level
    whole = oracle.detect(img.points, img.W, img.H, D, img.T)
    side = 1 << k
    rng = np.random.default_rng(100 + k)
    keep = (rng.random(2 * side * side) < 0.5).astype(np.uint8)
    part = oracle.detect_subtrees(img.points, img.W, img.H, D, img.T, k, keep)
    lv = whole.leaves
    sel = keep[lv[:, 0].astype(np.int64) * side * side + (lv[:, 1] >> (D - k)) * side + (lv[:, 2] >> (D - k))] == 1
    assert np.array_equal(part.leaves, lv[sel])
    assert np.array_equal(part.stats[:, :k], whole.stats[:, :k])
    assert np.array_equal(part.stats[:, k, [0, 2, 3]], whole.stats[:, k, [0, 2, 3]])
    assert np.all(part.stats[:, k, 1] <= whole.stats[:, k, 1])
