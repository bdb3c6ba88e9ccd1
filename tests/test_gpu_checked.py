"""The bounds-checked build (-DHHT_CHECKED): every index that the level kernel
takes from its data (parent and child record indices, cursors) is checked
against the current sizes, and a bad one sets an error status instead of
being used.  Run on the parity cases, this build is the out-of-bounds check
of the level kernel: it must report no error and give the oracle's results.  It runs in a child process because a process
loads one build of the library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import oracle, synth
from paper_1007_0547_gb300 import hht
assert "checked" in hht.version(), hht.version()
ctx = hht.Context(device=0)
imgs = [synth.plain_128(index=k) for k in range(3)]
imgs += [synth.random_small(53000 + s, max_side=300, max_n=2500, max_depth=9, max_T=12) for s in range(12)]
imgs += [synth.plain_1024()]
for im in imgs:
    got = ctx.detect(im.points, im.W, im.H, im.depth, im.T)
    want = oracle.detect(im.points, im.W, im.H, im.depth, im.T)
    assert np.array_equal(got.leaves_numpy(), want.leaves), im.name
    assert np.array_equal(got.stats, want.stats), im.name
batch = ctx.detect_batch([(im.points, im.W, im.H, im.depth, im.T) for im in imgs[:8]])
for im, r in zip(imgs[:8], batch):
    assert np.array_equal(r.leaves_numpy(), oracle.detect(im.points, im.W, im.H, im.depth, im.T).leaves), im.name
for shape in range(hht.TUNE_SHAPES):
    ctx.set_tuning(shape)
    im = imgs[-1]
    r = ctx.detect(im.points, im.W, im.H, im.depth, im.T)
    assert r.status == 0
print("checked ok")
'''


def test_checked_build_on_the_parity_cases():
    from paper_1007_0547_gb300 import build
    lib = build.build(extra_flags=["-DHHT_CHECKED"], variant="checked")
    env = dict(os.environ, HHT_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked ok" in r.stdout
