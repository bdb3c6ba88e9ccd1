"""Host-side logic of bench.py that needs no GPU: the parsing of the clock
samples that decide whether a run is kept, the source hash that guards the
recorded DRAM traffic, and the threaded CPU-oracle sample."""
import json
import os
import sys

import numpy as np

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, REPO)

import bench  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _parse(lines, tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = _Done()
    return s.stop()


def test_clock_samples_median_max_and_active_reasons(tmp_path):
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2040, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line",
            "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    got = _parse(rows, tmp_path)
    assert got["sm_mhz"] == 2040.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"] and got["samples"] == 3


def test_clock_samples_report_thermal_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 1300, 0x40, Not Active, Active, Not Active, Not Active"]
    assert _parse(rows, tmp_path)["reasons"] == ["hw_thermal_slowdown"]


def test_recorded_traffic_only_for_the_profiled_kernel_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"kernel_source_hash": bench.kernel_source_hash(), "dram_bytes_per_algorithmic_byte": 0.5}
    (prof / "pass_kernel_dram.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash reads the kernel sources under ROOT: point them at the real ones
    os.symlink(os.path.join(REPO, "paper_1007_0547_gb300"), tmp_path / "paper_1007_0547_gb300")
    assert bench.recorded_traffic() == 0.5
    rec["kernel_source_hash"] = "0" * 16
    (prof / "pass_kernel_dram.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic() is None


def test_threaded_oracle_sample_counts_every_test():
    imgs = [synth.random_small(500 + s, max_side=96, max_n=300, max_depth=6, max_T=5) for s in range(8)]
    tests, wall, cpu_s, threads, desc = bench.oracle_sample(imgs, cores=3)
    work = [len(im.points) * 2 ** im.depth for im in imgs]
    limit = max(work[k] for k in bench.CPU_SAMPLE)
    picks = [k for k in range(len(imgs)) if work[k] <= limit][: bench.CPU_IMAGES_PER_THREAD * 3]
    want = sum(oracle.detect(imgs[k].points, imgs[k].W, imgs[k].H, imgs[k].depth, imgs[k].T).total_tests()
               for k in picks)
    assert tests == want and threads == min(3, len(picks))
    assert wall > 0 and cpu_s > 0 and f"{len(picks)} batch images" in desc


def test_oracle_sample_of_one_image_runs_on_one_thread():
    im = synth.plain_128(index=0)
    tests, wall, cpu_s, threads, desc = bench.oracle_sample([im], cores=4)
    assert threads == 1 and tests == oracle.detect(im.points, im.W, im.H, im.depth, im.T).total_tests()
    assert desc.startswith(im.name)
    assert np.isfinite(wall)
