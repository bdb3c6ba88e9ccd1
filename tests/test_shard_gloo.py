"""Multi-rank sharding of a batch, on CPU with the gloo backend (world size 2).

Each rank detects its share of the images (the CPU oracle stands in for the
GPU here) and rank 0 gathers the results; the merged list must equal the
unsharded run image by image."""
import os
import socket

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
