"""ctypes binding of the C oracle (test infrastructure only).

detect() runs the depth-first hierarchy of Section 3 of the paper on one image
and returns its leaves (half, i, j, votes) in depth-first order (children NE,
NW, SW, SE; half 0 first) and per-level statistics
stats[half, level] = (regions tested, regions passed, votes, code evaluations).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hht_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

STAT_TESTED, STAT_PASSED, STAT_VOTES, STAT_TESTS = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


class _Leaf(ctypes.Structure):
    _fields_ = [("half", ctypes.c_uint32), ("i", ctypes.c_uint32), ("j", ctypes.c_uint32),
                ("votes", ctypes.c_uint32)]


class _Region(ctypes.Structure):
    _fields_ = [("half", ctypes.c_uint32), ("level", ctypes.c_uint32), ("i0", ctypes.c_uint32),
                ("j0", ctypes.c_uint32), ("size", ctypes.c_uint32), ("votes", ctypes.c_uint32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2) into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall", "-Wextra",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i16p = ctypes.POINTER(ctypes.c_int16)
            lib.oracle_detect.argtypes = [i16p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_Leaf), ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.POINTER(_Region), ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_int64)]
            lib.oracle_detect.restype = ctypes.c_int
            lib.oracle_getcode.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.c_int64, ctypes.c_int32]
            lib.oracle_getcode.restype = ctypes.c_uint32
            lib.oracle_scaled_F.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_int32]
            lib.oracle_scaled_F.restype = ctypes.c_int64
            lib.oracle_fht_votes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int64, ctypes.c_int64, ctypes.c_int32]
            lib.oracle_fht_votes.restype = ctypes.c_int
            lib.oracle_count_region.argtypes = [i16p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
            lib.oracle_count_region.restype = ctypes.c_int64
            lib.oracle_frame_side.argtypes = [ctypes.c_int32, ctypes.c_int32]
            lib.oracle_frame_side.restype = ctypes.c_int64
            _lib = lib
    return _lib


@dataclasses.dataclass
class OracleResult:
    leaves: np.ndarray   # uint32 [k, 4]: half, i, j, votes (depth-first order)
    stats: np.ndarray    # uint64 [2, depth + 1, 4]
    regions: Optional[np.ndarray] = None  # uint32 [r, 6]: half, level, i0, j0, size, votes
    rc: int = 0

    def total_tests(self) -> int:
        return int(self.stats[:, :, STAT_TESTS].sum())

    def total_votes(self) -> int:
        return int(self.stats[:, :, STAT_VOTES].sum())


def frame_side(W: int, H: int) -> int:
    return int(_load().oracle_frame_side(W, H))


def scaled_F(x: int, y: int, i: int, j: int, L: int, D: int) -> int:
    return int(_load().oracle_scaled_F(x, y, i, j, L, D))


def getcode(x: int, y: int, i0: int, j0: int, S: int, L: int, D: int) -> int:
    return int(_load().oracle_getcode(x, y, i0, j0, S, L, D))


def fht_votes(x: int, y: int, i0: int, j0: int, S: int, L: int, D: int) -> bool:
    return bool(_load().oracle_fht_votes(x, y, i0, j0, S, L, D))


def count_region(points: np.ndarray, W: int, H: int, depth: int, half: int, i0: int, j0: int, S: int) -> int:
    """Votes of one region counted directly over all points (no hierarchy)."""
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int16).reshape(-1, 2))
    return int(_load().oracle_count_region(pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), pts.shape[0],
                                           W, H, depth, half, i0, j0, S))


def detect(points: np.ndarray, W: int, H: int, depth: int, T: int, mode: str = "exact",
           dump_regions: bool = False, region_cap: int = 1 << 22) -> OracleResult:
    """Run the oracle; raises ValueError on argument/range errors."""
    lib = _load()
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int16).reshape(-1, 2))
    n = pts.shape[0]
    m = {"exact": 0, "fht": 1}[mode]
    stats = np.zeros((2, depth + 1, 4), dtype=np.uint64) if 1 <= depth <= 24 else np.zeros(8, np.uint64)
    nl = ctypes.c_int64(0)
    nr = ctypes.c_int64(0)
    regions = (_Region * region_cap)() if dump_regions else None
    cap = 1 << 16
    while True:
        leaves = (_Leaf * cap)()
        rc = lib.oracle_detect(pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), n, W, H, depth, T, m,
                               leaves, cap, ctypes.byref(nl),
                               stats.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                               regions, region_cap if dump_regions else 0, ctypes.byref(nr))
        if rc == -4:
            cap = int(nl.value) + 1
            continue
        break
    if rc == -1:
        raise ValueError("oracle: bad argument")
    if rc == -2:
        raise ValueError("oracle: point outside the image")
    if rc != 0:
        raise RuntimeError(f"oracle failed with code {rc}")
    k = int(nl.value)
    lv = np.frombuffer(leaves, dtype=np.uint32).reshape(-1, 4)[:k].copy()
    reg = None
    if dump_regions:
        r = min(int(nr.value), region_cap)
        reg = np.frombuffer(regions, dtype=np.uint32).reshape(-1, 6)[:r].copy()
        if int(nr.value) > region_cap:
            raise RuntimeError("oracle: region dump capacity exceeded")
    return OracleResult(lv, stats, reg, rc)
