#!/usr/bin/env python
"""Benchmark: line x region tests per second of the hierarchical Hough
transform on the 256-image mixed batch (side log-uniform in 256-2048, 8-64
segments, 0.5-5% noise, depth ceil(log2 side), T = 2*side/32), batched through
one context on one GB300 per rank.

One step = one hht_detect_batch() call over the whole batch (every level of
every image, both halves, leaves sorted and copied out).  Prints one JSON line
on rank 0.  `--impl reference` times the CPU oracle instead (rank 0 only).

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 use
torch.distributed.run with one process per GPU (weak scaling: each rank runs
its own 256 images).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "line×region tests/s"
UNIT = "tests/s"
WORKLOADS = {
    "batch_256": "256 images, side log-uniform 256-2048, 8-64 segments, noise 0.5-5%, depth ceil(log2 side), "
                 "T = 2*side/32, both halves",
    "plain_1024": "1024x1024, 32 segments of 100-1000 px, 2% noise, depth 10, T = 64, both halves",
    "plain_4096": "4096x4096, 512 segments of 50-4000 px, 1% noise, depth 12, T = 128, both halves",
    "plain_128": "128x128, 4 segments, 1% noise, depth 7, T = 20, both halves",
}
CPU_SAMPLE = [0, 1]   # batch images timed on the CPU oracle (sides 334 and 552)
CPU_IMAGES_PER_THREAD = 2  # the all-cores oracle sample: this many batch images per host thread


def load_images(workload: str, rank: int):
    if workload == "batch_256":
        return synth.batch_256(256, first=256 * rank)
    fn = {"plain_1024": synth.plain_1024, "plain_4096": synth.plain_4096, "plain_128": synth.plain_128}[workload]
    return [fn(index=rank)]


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the level (pass) kernel's source: its section of hht_kernels.cu
    (from the pass banner to the next one) and the device helpers it uses."""
    csrc = os.path.join(ROOT, "paper_1007_0547_gb300", "csrc")
    with open(os.path.join(csrc, "hht_kernels.cu"), "rb") as f:
        src = f.read()
    start = src.index(b"// " + b"=" * 76 + b" pass")
    end = src.index(b"// " + b"=" * 76, start + 10)
    h = hashlib.sha256()
    h.update(src[start:end])
    with open(os.path.join(csrc, "hht_device.cuh"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per algorithmic byte of the pass kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "pass_kernel_dram.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    return float(d["dram_bytes_per_algorithmic_byte"])


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="hht_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores() -> int:
    """Host threads this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _oracle_one(job):
    """One oracle detection; its tests and the CPU seconds of the thread that
    ran it (ctypes releases the GIL while the C oracle runs)."""
    import oracle
    im, pts = job
    t = time.thread_time()
    r = oracle.detect(pts, im.W, im.H, im.depth, im.T)
    return r.total_tests(), time.thread_time() - t


def oracle_sample(images, cores=None):
    """Time the CPU oracle, as it stands, on a bounded sample of the workload,
    one image per host thread at a time.  A batch's sample is its first
    CPU_IMAGES_PER_THREAD images per thread whose work (n * 2^depth) is at
    most that of the larger of the CPU_SAMPLE images; a single large image is
    stood in for by a horizontal band of its rows, on one thread.  Returns
    (tests, wall seconds, thread CPU seconds, threads used, description)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    oracle.build()
    if len(images) > 1:
        work = [len(im.points) * 2 ** im.depth for im in images]
        limit = max(work[k] for k in CPU_SAMPLE if k < len(images))
        cores = max(1, cores or host_cores())
        picks = [k for k in range(len(images)) if work[k] <= limit][: CPU_IMAGES_PER_THREAD * cores]
        jobs = [(images[k], images[k].points) for k in picks]
        desc = (f"{len(picks)} batch images with n * 2^depth <= {limit} (indices {picks[0]}..{picks[-1]}), "
                f"one per thread at a time")
    else:
        im = images[0]
        pts = im.points if im.n <= 60000 else im.points[im.points[:, 1] < max(1, im.H // 16)]
        jobs = [(im, pts)]
        desc = f"{im.name}(side {im.W}, n {len(pts)})"
    threads = min(max(1, cores or host_cores()), len(jobs))
    with ThreadPoolExecutor(max_workers=threads) as ex:
        t = time.perf_counter()
        outs = list(ex.map(_oracle_one, jobs))
        wall = time.perf_counter() - t
    return sum(o[0] for o in outs), wall, sum(o[1] for o in outs), threads, desc


def run_reference(args, rank):
    if rank != 0:
        return
    images = load_images(args.workload, 0)
    for _ in range(args.warmup):
        oracle_sample(images)
    tests = secs = cpu_s = 0.0
    sample, threads = "", 1
    for _ in range(args.steps):
        t, s, c, threads, sample = oracle_sample(images)
        tests += t
        secs += s
        cpu_s += c
    v = tests / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                                            "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "per_thread_value": tests / cpu_s if cpu_s > 0 else None},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_front_end(args, rank):
    """The front-end kernel alone (hht_edges: Sobel's operator and the
    ALPHA/BETA split) on the 4096x4096 grey image, image resident on the
    device; device time from the library's own events."""
    import torch
    from paper_1007_0547_gb300 import build as hbuild
    hbuild.build()
    from paper_1007_0547_gb300 import hht
    if rank != 0:
        return
    g = synth.gray_4096()
    img = torch.from_numpy(g.pixels).cuda()
    ctx = hht.Context(device=0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        a, b = ctx.edges(img, g.threshold)
    torch.cuda.synchronize()
    ctx.profile(True)
    for _ in range(args.steps):
        flush.zero_()
        a, b = ctx.edges(img, g.threshold)
    p = ctx.profile_read()
    ctx.profile(False)
    ms = p["edges_ms"] / max(1, p["edges_launches"])
    pts = int(len(a) + len(b))
    byt = g.W * g.H + 4 * pts
    peak, peak_kind = read_peaks()
    print(json.dumps({"metric": "pixels/s (Sobel and ALPHA/BETA split)", "value": g.W * g.H / (ms / 1e3),
                      "unit": "pixels/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": "u8", "data": "synthetic",
                      "config": {"workload": "gray_4096", "threshold": g.threshold, "edge_points": pts},
                      "roofline": {"kernel": "edges_kernel", "bound": "alu", "algorithmic_bytes": byt,
                                   "hbm_achieved_GBps": byt / (ms / 1e3) / 1e9, "hbm_peak": peak,
                                   "hbm_frac": byt / (ms / 1e3) / 1e9 / peak, "peak_source": f"{peak_kind} hbm_gbs"}}),
          flush=True)
    ctx.close()


def serving_leg(ctx, n_requests: int, load: float):
    """Open-loop Poisson stream of `n_requests` serving requests through
    hht_submit / hht_progress / hht_done_tickets / hht_poll (continuous
    batching) on `ctx`.  Rate = `load` x the saturated request rate measured
    first on the same requests.  Returns the latency / throughput record."""
    import torch
    reqs = synth.serving_requests(n_requests)

    def drain(arrivals):
        """Submit request k at arrivals[k] (s after start); return per-request
        (arrival, done) wall times and the total time."""
        n = len(reqs)
        t_arr = [0.0] * n
        t_done = [0.0] * n
        tickets = {}
        k = 0
        done = 0
        t0 = time.perf_counter()
        while done < n:
            now = time.perf_counter() - t0
            while k < n and arrivals[k] <= now:
                im = reqs[k]
                tickets[ctx.submit(im.points, im.W, im.H, im.depth, im.T)] = k
                t_arr[k] = arrivals[k]
                k += 1
            if tickets:
                ctx.progress()
                now = time.perf_counter() - t0
                for t in ctx.done_tickets():  # only finished requests are polled
                    j = tickets.pop(t)
                    if ctx.poll(t) is None:
                        raise RuntimeError("a listed ticket was still pending")
                    t_done[j] = now
                    done += 1
            elif k < n:
                time.sleep(max(0.0, min(0.01, arrivals[k] - now)))
        return t_arr, t_done, time.perf_counter() - t0

    # warm-up on a few requests, then the saturated rate (everything at t = 0)
    for im in reqs[:8]:
        ctx.detect(im.points, im.W, im.H, im.depth, im.T)
    torch.cuda.synchronize()
    _, _, sat_s = drain([0.0] * len(reqs))
    sat_rate = len(reqs) / sat_s
    rate = load * sat_rate
    arrivals = list(synth.poisson_arrivals(len(reqs), rate))
    t_arr, t_done, total_s = drain(arrivals)
    per = [((d - a) * 1e3, im) for a, d, im in zip(t_arr, t_done, reqs)]
    lat = sorted(x for x, _ in per)

    def pct(xs, q):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, int(q * len(xs)))] if xs else None

    small = [x for x, im in per if im.W <= 1024]
    large = [x for x, im in per if im.W > 1024]
    slowest = sorted(per, key=lambda t: -t[0])[:3]
    return {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "side_le_1024": {"requests": len(small), "p50_ms": pct(small, 0.5), "p99_ms": pct(small, 0.99)},
            "side_gt_1024": {"requests": len(large), "p50_ms": pct(large, 0.5), "p99_ms": pct(large, 0.99)},
            "slowest": [{"ms": round(x, 2), "side": im.W, "n": im.n, "depth": im.depth, "T": im.T} for x, im in slowest],
            "images_per_s": len(reqs) / total_s, "saturated_images_per_s": sat_rate,
            "offered_rate_per_s": rate, "load": load, "requests": len(reqs),
            "description": "side log-uniform 64-4096, 1-256 segments, noise 0-3%, depth ceil(log2 side), "
                           "T uniform 16-256; Poisson arrivals; latency = done - arrival (wall clock)"}


def single_image_latency(ctx, runs: int = 30):
    """Wall-clock latency of one hht_detect call (points resident on the
    device, leaves into a device buffer) on the 128x128 and 1024x1024
    workloads, after warm-up: p50 / p99 over `runs` calls."""
    import torch
    out = {}
    for name, fn in (("plain_128", synth.plain_128), ("plain_1024", synth.plain_1024)):
        im = fn()
        pts = torch.from_numpy(im.points).cuda()
        for _ in range(5):
            ctx.detect(pts, im.W, im.H, im.depth, im.T)
        torch.cuda.synchronize()
        ts = []
        for _ in range(runs):
            t0 = time.perf_counter()
            ctx.detect(pts, im.W, im.H, im.depth, im.T)
            ts.append((time.perf_counter() - t0) * 1e3)
        ts.sort()
        out[name] = {"p50_ms": ts[len(ts) // 2], "p99_ms": ts[min(len(ts) - 1, int(0.99 * len(ts)))],
                     "runs": runs, "n": im.n}
    return out


def run_ncu_case(args, rank):
    """One small detection for an ncu capture.  removal1024: the solution()
    walk of the 1024x1024 image.  batch8: the pass kernel on 8 images of
    the 256-image batch (indices 0, 32, ..., 224), level form (one launch per
    pass), tile shape --tile-shape.  Prints, per pass launch s, the records it
    reads (the level s-1 stream) and writes (the level s stream), from the
    detection's statistics: a level's tests are four per voter of a passed
    parent, and a unit keeps lists of its levels up to depth - 2."""
    from paper_1007_0547_gb300 import build as hbuild
    hbuild.build()
    from paper_1007_0547_gb300 import hht
    import torch
    if rank != 0:
        return
    if args.ncu_case == "removal1024":
        # the solution() walk of the 1024x1024 image, once (one removal_kernel launch)
        im = synth.plain_1024()
        ctx = hht.Context(device=0)
        res, _ = ctx.detect_removal(torch.from_numpy(im.points).cuda(), im.W, im.H, im.depth, im.T,
                                    with_plotted=False)
        torch.cuda.synchronize()
        print(json.dumps({"case": "removal1024", "n": im.n, "depth": im.depth, "T": im.T,
                          "accepted_cells": int(res.n_leaves), "code_tests": int(res.total_tests())}), flush=True)
        ctx.close()
        return
    imgs = [synth.batch_image(k) for k in range(0, 256, 32)]
    dev = [(torch.from_numpy(im.points).cuda(), im.W, im.H, im.depth, im.T) for im in imgs]
    ctx = hht.Context(device=0)
    ctx.set_batch_mode(hht.BATCH_LEVELS)
    ctx.set_tuning(args.tile_shape)
    res = ctx.detect_batch(dev)
    torch.cuda.synchronize()
    dmax = max(im.depth for im in imgs)
    launches = []
    for s in range(1, dmax):
        rd = sum(int(r.stats[h, s, 3]) // 4 for r, im in zip(res, imgs) for h in range(2) if s - 1 <= im.depth - 2)
        wr = sum(int(r.stats[h, s + 1, 3]) // 4 for r, im in zip(res, imgs) for h in range(2) if s <= im.depth - 2)
        if rd > 0:  # the level form launches no pass over an empty stream
            launches.append({"launch": len(launches) + 1, "pass": s, "records_read": rd, "records_written": wr,
                             "algorithmic_bytes": 8 * (rd + wr)})
    print(json.dumps({"case": "batch8", "images": [k for k in range(0, 256, 32)],
                      "sides": [im.W for im in imgs], "depths": [im.depth for im in imgs],
                      "tile_shape": args.tile_shape, "pass_launches": launches}), flush=True)
    ctx.close()


def run_serving(args, rank):
    """The serving leg alone, at --serve-requests and --serve-load."""
    from paper_1007_0547_gb300 import build as hbuild
    hbuild.build()
    from paper_1007_0547_gb300 import hht
    if rank != 0:
        return
    ctx = hht.Context(device=0)
    leg = serving_leg(ctx, args.serve_requests, args.serve_load)
    line = {"metric": "serving latency p50/p99 (ms) and images/s", "value": leg["p50_ms"], "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic", **leg,
            "config": {"workload": "serving", "requests": leg["requests"], "description": leg["description"]}}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="batch_256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-persistent", "--no-levels", dest="no_persistent", action="store_true",
                    help="skip the level-form comparison")
    ap.add_argument("--no-fht", action="store_true", help="skip the prior-art FHT circle-test comparison")
    ap.add_argument("--no-front-end", action="store_true", help="skip the front-end and line-extraction timings")
    ap.add_argument("--no-removal", action="store_true", help="skip the solution() (voter removal) timing")
    ap.add_argument("--no-latency", action="store_true",
                    help="skip the single-image latency (128x128, 1024x1024) and serving legs of the default line")
    ap.add_argument("--leg-requests", type=int, default=200,
                    help="requests of the serving leg in the default line")
    ap.add_argument("--serve", action="store_true", help="open-loop serving benchmark instead of the batch line")
    ap.add_argument("--front-end", action="store_true",
                    help="time only the front-end kernel (Sobel and split) on the 4096x4096 grey image")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-load", type=float, default=0.8, help="offered rate as a fraction of the saturated rate")
    ap.add_argument("--ncu-case", choices=["batch8", "removal1024"],
                    help="run one small detection for an ncu capture (of the pass kernel: batch8; of the "
                         "solution() walk: removal1024) and exit")
    ap.add_argument("--tile-shape", type=int, default=0, help="pass tile shape of --ncu-case")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.ncu_case:
        run_ncu_case(args, rank)
        return
    if args.serve:
        run_serving(args, rank)
        return
    if args.front_end:
        run_front_end(args, rank)
        return

    import torch
    import torch.distributed as dist
    from paper_1007_0547_gb300 import build as hbuild
    if rank == 0 or world == 1:
        hbuild.build()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
        dist.barrier()
        hbuild.build()  # no-op once rank 0 has built
    from paper_1007_0547_gb300 import hht

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    images = load_images(args.workload, rank)
    dev_images = [(torch.from_numpy(im.points).to(dev), im.W, im.H, im.depth, im.T) for im in images]
    host_images = [(np.ascontiguousarray(im.points), im.W, im.H, im.depth, im.T) for im in images]
    stream = torch.cuda.current_stream(dev)
    ctx = hht.Context(device=local, stream=stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)  # 512 MB > 129 MB L2

    def step():
        if len(dev_images) == 1:
            return [ctx.detect(*dev_images[0])]
        return ctx.detect_batch(dev_images)

    # the first call of the fresh context: sizes from upper bounds, one CUDA
    # graph captured and launched (wall clock, allocations included)
    ctx.profile(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step()
    torch.cuda.synchronize()
    fp = ctx.profile_read()
    first_call = {"ms": (time.perf_counter() - t0) * 1e3, "graph_launches": int(fp["graph_launches"]),
                  "graph_captures": int(fp["graph_captures"]), "graph_fallbacks": int(fp["graph_fallbacks"]),
                  "what": "first detection call of a new context on this workload (wall clock; device memory "
                          "allocated and the level loop's CUDA graph captured inside it)"}
    ctx.profile(False)

    tuning = None
    if not args.no_autotune:
        # tile shape of the level kernel for this workload (cached per device and workload class)
        shape, times = ctx.autotune(dev_images, cache=os.environ.get("HHT_TUNE_CACHE"))
        tuning = {"shape": shape, "pass_ms_per_shape": times}
    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    tests_per_step = sum(r.total_tests() for r in res)
    leaves_per_step = sum(r.n_leaves for r in res)

    # ---------------------------------------------------------------- timed region
    phys = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis:
        ids = [v.strip() for v in vis.split(",")]
        if local < len(ids) and ids[local].isdigit():
            phys = int(ids[local])
    sampler = ClockSampler(phys)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # profiling adds event records to the captured graph: capture that graph
    # in an untimed step, then reset the counters for the timed steps
    ctx.profile(True)
    step()
    torch.cuda.synchronize()
    ctx.profile(True)
    sampler.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    prof = ctx.profile_read()
    ctx.profile(False)
    total_ms = sum(times)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        n = torch.tensor([tests_per_step], dtype=torch.float64, device=dev)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        tests_all = float(n.item())
        dist.barrier()
    else:
        tests_all = float(tests_per_step)
    value = tests_all * args.steps / (total_ms / 1e3)
    images_per_s = len(images) * world * args.steps / (total_ms / 1e3)

    # ---------------------------------------------------------------- end to end (host buffers)
    e2e = None
    if not args.no_e2e:
        h2d = sum(im.n for im in images) * 4
        d2h = leaves_per_step * 16 + len(images) * (2 * 25 * 4 * 8)
        # the inputs and the leaves live in pinned host memory (allocated once,
        # outside the timed region); every step copies the points in and all
        # leaves and statistics out
        pinned_images = [(torch.from_numpy(p).pin_memory(), W, H, D, T) for (p, W, H, D, T) in host_images]
        leaves_host = torch.empty((max(leaves_per_step, 1), 4), dtype=torch.int32, pin_memory=True)

        def e2e_step():
            if len(pinned_images) == 1:
                ctx.detect(*pinned_images[0], leaves_out=leaves_host)
            else:
                ctx.detect_batch(pinned_images, leaves_out=leaves_host)

        for _ in range(args.warmup):
            e2e_step()
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            ts.append(time.perf_counter() - t0)
        e2e_s = sum(ts)
        if world > 1:
            t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": tests_all * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * e2e_s / args.steps,
               "ms_steps": [round(1e3 * t, 2) for t in ts]}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---------------------------------------------------------------- per-image launch sequence
    per_image = None
    if len(dev_images) > 1:
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for x in dev_images:
            ctx.detect(*x)
        e1.record(stream)
        e1.synchronize()
        seq_ms = e0.elapsed_time(e1)
        per_image = {"images_per_s": len(dev_images) / (seq_ms / 1e3),
                     "tests_per_s": tests_per_step / (seq_ms / 1e3), "ms": seq_ms}

    # ---------------------------------------------------------------- level form (host-driven, one sync per level)
    levels = None
    if not args.no_persistent:
        ctx.set_batch_mode(hht.BATCH_LEVELS)
        step()  # allocations
        torch.cuda.synchronize()
        lv_ms = []
        for _ in range(max(2, args.steps // 2)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            lv_ms.append(e0.elapsed_time(e1))
        ctx.set_batch_mode(hht.BATCH_GRAPH)
        lm = sum(lv_ms) / len(lv_ms)
        levels = {"what": "the same detection in the level form: one selection and one pass launch per level with "
                          "a host synchronisation each, buffers sized exactly",
                  "ms_per_step": lm, "images_per_s": len(dev_images) / (lm / 1e3),
                  "tests_per_s": tests_per_step / (lm / 1e3)}

    # ---------------------------------------------------------------- prior-art FHT circle test, same images
    fht = None
    if not args.no_fht:
        votes_exact = sum(int(r.stats[:, :, 2].sum()) for r in res)
        ctx.set_predicate(hht.PREDICATE_FHT)
        fres = step()  # allocations
        torch.cuda.synchronize()
        f_ms = []
        for _ in range(max(2, args.steps // 2)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fres = step()
            e1.record(stream)
            e1.synchronize()
            f_ms.append(e0.elapsed_time(e1))
        ctx.set_predicate(hht.PREDICATE_EXACT)
        fm = sum(f_ms) / len(f_ms)
        votes_fht = sum(int(r.stats[:, :, 2].sum()) for r in fres)
        fht = {"what": "circumscribed-circle test of the prior-art FHT (exact integer form), same images and thresholds",
               "ms_per_step": fm, "tests_per_s": sum(r.total_tests() for r in fres) / (fm / 1e3),
               "votes": votes_fht, "votes_exact": votes_exact, "C_v": votes_fht / max(1, votes_exact),
               "C_t": fm / (total_ms / args.steps), "leaves": int(sum(r.n_leaves for r in fres))}

    # ---------------------------------------------------------------- front end and lines (4096^2 grey image)
    front = None
    if not args.no_front_end and rank == 0:
        g = synth.gray_4096()
        gimg = torch.from_numpy(g.pixels).to(dev)
        for _ in range(3):
            ctx.edges(gimg, g.threshold)
        torch.cuda.synchronize()
        ctx.profile(True)
        for _ in range(5):
            flush.zero_()
            ea, eb = ctx.edges(gimg, g.threshold)
        fp = ctx.profile_read()
        ctx.profile(False)
        e_ms = fp["edges_ms"] / max(1, fp["edges_launches"])
        e_bytes = g.W * g.H + 4 * (len(ea) + len(eb))
        d_ms, l_ms = [], []
        for _ in range(3):
            flush.zero_()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            dres = ctx.detect_image(gimg, g.threshold, g.depth, g.T)
            e1.record(stream)
            glines = ctx.lines(0)
            e2.record(stream)
            e2.synchronize()
            d_ms.append(e0.elapsed_time(e1))
            l_ms.append(e1.elapsed_time(e2))
        front = {"workload": "gray_4096 (4096x4096 grey image, Sobel threshold 200, depth 12, T = 128)",
                 "edges_kernel_ms": e_ms, "edges_points": int(len(ea) + len(eb)),
                 "edges_algorithmic_GBps": e_bytes / (e_ms / 1e3) / 1e9,
                 "edges_hbm_frac": e_bytes / (e_ms / 1e3) / 1e9 / read_peaks()[0],
                 "detect_image_ms": min(d_ms), "detect_image_tests": int(dres.total_tests()),
                 "leaves": int(dres.n_leaves), "lines_ms": min(l_ms), "lines": int(len(glines))}

    # ---------------------------------------------------------------- solution() traversal, same images
    removal = None
    if not args.no_removal and rank == 0:
        ctx.detect_removal_batch(dev_images)  # allocations
        torch.cuda.synchronize()
        r_ms = []
        for _ in range(2):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rres = ctx.detect_removal_batch(dev_images)
            e1.record(stream)
            e1.synchronize()
            r_ms.append(e0.elapsed_time(e1))
        rm = min(r_ms)
        rtests = sum(r.total_tests() for r in rres)
        removal = {"what": "depth-first traversal with the paper's solution() step (voters of accepted cells removed "
                           "from later regions); one block of four warps per image and half",
                   "ms_per_step": rm, "tests_per_s": rtests / (rm / 1e3), "images_per_s": len(dev_images) / (rm / 1e3),
                   "accepted_cells": int(sum(r.n_leaves for r in rres))}

    # ---------------------------------------------------------------- single images and serving (configs 1, 2, 5)
    # the batch context's buffers (sized from the batch's upper bounds) are
    # given back first, so that the serving leg's memory budget is the
    # device's, as for a serving process of its own
    ctx.close()
    latency, serving = None, None
    if not args.no_latency and rank == 0:
        lctx = hht.Context(device=local, stream=stream)
        latency = single_image_latency(lctx)
        lctx.close()
        sctx = hht.Context(device=local)
        serving = serving_leg(sctx, args.leg_requests, args.serve_load)
        sctx.close()

    # ---------------------------------------------------------------- roofline of the pass kernel
    peak, peak_kind = read_peaks()
    achieved = (prof["pass_bytes"] / 1e9) / (prof["pass_ms"] / 1e3) if prof["pass_ms"] > 0 else 0.0
    ratio = recorded_traffic()
    per_launch = prof["pass_bytes"] / max(1, prof["pass_launches"])
    roofline = {"kernel": "pass_kernel<int32_t>", "bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                "traffic": (ratio * per_launch) if ratio is not None else None,
                "algorithmic_bytes_per_launch": per_launch,
                "launches": prof["pass_launches"], "pass_ms_per_step": prof["pass_ms"] / args.steps,
                "select_ms_per_step": prof["select_ms"] / args.steps,
                "stage_ms_per_step": prof["stage_ms"] / args.steps}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        t, s, c, threads, sample = oracle_sample(images)
        cpu = {"value": t / s, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
               "seconds": s, "per_thread_value": t / c if c > 0 else None}

    srt = sorted(times)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload],
                   "images_per_rank": len(images), "points_per_rank": int(sum(im.n for im in images)),
                   "tests_per_step_per_rank": int(tests_per_step), "leaves_per_step_per_rank": int(leaves_per_step),
                   "l2": "512 MB buffer written between timed steps; voter streams are larger than L2"},
        "images_per_s": images_per_s,
        "latency_ms": {"p50": srt[len(srt) // 2], "p99": srt[min(len(srt) - 1, int(0.99 * len(srt)))],
                       "what": "one step (whole batch)"},
        "per_image_sequence": per_image,
        "execution_form": {"headline": "graph: the whole level loop of a step is one CUDA-graph launch (stage, "
                                       "then selection and pass per level, sizes read on the device), one host "
                                       "synchronisation per step",
                           "graph_launches_timed": int(prof["graph_launches"]),
                           "graph_captures_timed": int(prof["graph_captures"]),
                           "graph_fallbacks_timed": int(prof["graph_fallbacks"])},
        "first_call": first_call,
        "levels_form": levels,
        "fht_form": fht,
        "front_end": front,
        "removal_form": removal,
        "single_image_latency": latency,
        "serving": serving,
        "e2e": e2e,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": int(prof["launches"]),
        "autotune": tuning,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
