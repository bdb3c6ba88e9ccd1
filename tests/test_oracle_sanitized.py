"""The oracle's pins again, with the oracle's C code built under AddressSanitizer
and UBSan: an out-of-bounds access, a use after free, a signed overflow or a
bad shift anywhere in the oracle stops the run with a report.

The pins run in a child pytest that preloads libasan (Python itself is not
instrumented) and selects the sanitized build through $HHT_ORACLE_VARIANT."""
import os
import subprocess
import sys

import pytest

import oracle

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_front_end.py", "tests/test_oracle_lines.py",
             "tests/test_oracle_removal.py"]


def _libasan():
    try:
        path = subprocess.check_output(["gcc", "-print-file-name=libasan.so"], text=True).strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_oracle_pins_pass_under_address_and_undefined_behaviour_sanitizers():
    asan = _libasan()
    if asan is None:
        pytest.skip("gcc has no AddressSanitizer runtime here")
    try:
        lib = oracle.build(variant="sanitized")
    except subprocess.CalledProcessError:
        pytest.skip("gcc cannot build with -fsanitize=address,undefined here")
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1", HHT_ORACLE_VARIANT="sanitized")
    # the child really loads the sanitized library
    probe = subprocess.run([sys.executable, "-c", "import oracle, numpy as np; "
                            "oracle.detect(np.zeros((1, 2), np.int16), 4, 4, 2, 1); print(oracle.loaded_path())"],
                           cwd=REPO, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0, probe.stderr[-3000:]
    assert os.path.samefile(probe.stdout.strip().splitlines()[-1], lib)
    run = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                          *PIN_FILES], cwd=REPO, env=env, capture_output=True, text=True, timeout=900)
    assert run.returncode == 0, run.stdout[-4000:] + run.stderr[-4000:]
    assert "passed" in run.stdout
