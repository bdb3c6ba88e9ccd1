"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle/hht_oracle.c, builds it with
gcc, and runs a fast subset of the oracle's pins against that build in a child
process ($HHT_ORACLE_LIB); the subset must fail.  A control build of the
unchanged source must pass the same subset, so that a broken harness cannot
pass for a caught mistake.  Nothing here touches a GPU."""
import os
import subprocess
import sys

import pytest

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(REPO, "oracle", "hht_oracle.c")
PINS = "tests/test_oracle_pins.py"
PIN_SUBSET = ("hand or concurrency_vertex or brute_force_small or fht_brute_force_tiny or stats_identities "
              "or transpose or leaves_come")
FRONT_END = "tests/test_oracle_front_end.py"
REMOVAL = "tests/test_oracle_removal.py"
LINES = "tests/test_oracle_lines.py"

# (name, text in the source, its replacement, occurrences to replace (0 = all), pin file, -k subset)
MUTANTS = [
    ("a corner on the line counted as below (<= for <)", ") < 0) code |=", ") <= 0) code |=", 0, PINS, PIN_SUBSET),
    ("NE and NW bits swapped", "code |= 8u; /* bit 1: NorthEast */", "code |= 4u; /* bit 1: NorthEast */", 1,
     PINS, PIN_SUBSET),
    ("the -K*y term of K*F dropped", "return K_b - slope * K_m - K * intercept;", "return K_b - slope * K_m;", 1,
     PINS, PIN_SUBSET),
    ("a region passes only above T (> for >=)", "if (kept && cnt >= w->T)", "if (kept && cnt > w->T)", 1,
     PINS, PIN_SUBSET),
    ("leaf i and j transposed", "lf->i = (uint32_t)ci[q]; lf->j = (uint32_t)cj[q];",
     "lf->i = (uint32_t)cj[q]; lf->j = (uint32_t)ci[q];", 1, PINS, PIN_SUBSET),
    ("half 1 not swapped", "px[k] = half == 0 ? xy[2 * k] : xy[2 * k + 1];\n"
                           "            py[k] = half == 0 ? xy[2 * k + 1] : xy[2 * k];",
     "px[k] = xy[2 * k];\n            py[k] = xy[2 * k + 1];", 1, PINS, PIN_SUBSET),
    ("NW and SW children exchanged", "const int64_t cj[4] = {j0 + h, j0 + h, j0, j0};",
     "const int64_t cj[4] = {j0 + h, j0, j0 + h, j0};", 1, PINS, PIN_SUBSET),
    ("three codes counted per parent voter", "*stat_at(w, child, 3) += 4 * (uint64_t)nV;",
     "*stat_at(w, child, 3) += 3 * (uint64_t)nV;", 1, PINS, PIN_SUBSET),
    ("FHT circle radius S/2 instead of S/sqrt(2)", "const __int128 rhs = (__int128)2 * S * S *",
     "const __int128 rhs = (__int128)1 * S * S *", 1, PINS, PIN_SUBSET),
    ("Sobel centre weight 1 instead of 2", "*gx = (P(1, -1) + 2 * P(1, 0) + P(1, 1))",
     "*gx = (P(1, -1) + P(1, 0) + P(1, 1))", 1, FRONT_END, None),
    ("gradient ties |gx| = |gy| sent to BETA", "if (ax <= ay) {", "if (ax < ay) {", 1, FRONT_END, None),
    ("edge only above the threshold (> for >=)", "(int64_t)gy * gy < t2) continue;",
     "(int64_t)gy * gy <= t2) continue;", 1, FRONT_END, None),
    ("solution() plots nothing", "for (int64_t k = 0; k < cnt; ++k) r->removed[buf[k]] = 1;", "", 1, REMOVAL, None),
    ("removed points still counted as tested",
     "if (r->removed[V[k]]) continue; /* its codes were zeroed by an earlier solution() */\n            ++evaluated;",
     "++evaluated;\n            if (r->removed[V[k]]) continue;", 1, REMOVAL, None),
    ("subtree keep mask read transposed", "+ (ci[q] / h) * side + cj[q] / h] != 0;",
     "+ (cj[q] / h) * side + ci[q] / h] != 0;", 1, "tests/test_shard_gloo.py", "one_shard"),
    ("lines: centre sums not weighted by votes",
     "L->sum_i2 += (uint64_t)leaves[k].votes * (2u * (uint64_t)leaves[k].i + 1u);",
     "L->sum_i2 += (2u * (uint64_t)leaves[k].i + 1u);", 1, LINES, None),
    ("lines: peak ties go to the later leaf", "if (leaves[k].votes > L->votes) {", "if (leaves[k].votes >= L->votes) {",
     1, LINES, None),
    ("lines: 4-neighbourhood instead of 8", "if (di < -1 || di > 1 || dj < -1 || dj > 1) continue;",
     "if (di < -1 || di > 1 || dj < -1 || dj > 1 || (di != 0 && dj != 0)) continue;", 1, LINES, None),
]


def _build(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    lib = tmp_path / f"{name}.so"
    src.write_text(text)
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-o", str(lib), str(src)])
    return str(lib)


def _run_pins(lib, pins, subset):
    env = dict(os.environ, HHT_ORACLE_LIB=lib)
    env.pop("HHT_ORACLE_VARIANT", None)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu", pins]
    if subset:
        cmd += ["-k", subset]
    return subprocess.run(cmd, cwd=REPO, env=env, capture_output=True, text=True, timeout=600)


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("pins,subset", sorted({(m[4], m[5]) for m in MUTANTS}, key=str))
def test_control_build_passes(source, tmp_path, pins, subset):
    run = _run_pins(_build(tmp_path, "control", source), pins, subset)
    assert run.returncode == 0, run.stdout[-3000:] + run.stderr[-3000:]


@pytest.mark.parametrize("name,old,new,count,pins,subset", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(source, tmp_path, name, old, new, count, pins, subset):
    assert old in source, f"mutation site not found: {name}"
    text = source.replace(old, new) if count == 0 else source.replace(old, new, count)
    assert text != source
    run = _run_pins(_build(tmp_path, "mutant", text), pins, subset)
    assert run.returncode == 1, f"{name}: pins did not fail\n" + run.stdout[-2000:] + run.stderr[-2000:]
