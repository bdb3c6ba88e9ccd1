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


# Flags of the "sanitized" variant: AddressSanitizer and UBSan, stopping at the
# first undefined behaviour.  A process that loads it must preload libasan.
_SANITIZED_FLAGS = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined",
                    "-fno-omit-frame-pointer"]


def build(force: bool = False, variant: Optional[str] = None) -> str:
    """Compile the oracle with gcc (plain C11) into oracle/_build/: -O2 by
    default; variant "sanitized" (or $HHT_ORACLE_VARIANT=sanitized) builds it
    with AddressSanitizer and UBSan instead."""
    variant = variant if variant is not None else os.environ.get("HHT_ORACLE_VARIANT", "")
    if variant not in ("", "sanitized"):
        raise ValueError(f"unknown oracle variant {variant!r}")
    path = _LIB_PATH if not variant else os.path.join(_OUT_DIR, f"liboracle_{variant}.so")
    flags = ["-O2"] if not variant else _SANITIZED_FLAGS
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(path)) or os.path.getmtime(path) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *flags, "-std=gnu11", "-fPIC", "-shared", "-Wall", "-Wextra",
                               "-o", tmp, _SRC])
        os.replace(tmp, path)
    return path


def loaded_path() -> str:
    """Path of the oracle library this process loaded."""
    return _load()._name


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # $HHT_ORACLE_LIB names a prebuilt oracle library (the tests load
            # deliberately broken builds this way to check that the pins fail)
            lib = ctypes.CDLL(os.environ.get("HHT_ORACLE_LIB") or build())
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
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_sobel.argtypes = [u8p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         i32p, i32p]
            lib.oracle_sobel.restype = None
            lib.oracle_edges.argtypes = [u8p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, i16p, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64), i16p, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64)]
            lib.oracle_edges.restype = ctypes.c_int
            lib.oracle_detect_subtrees.argtypes = [i16p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(_Leaf),
                                                   ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                                   ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_detect_subtrees.restype = ctypes.c_int
            lib.oracle_detect_removal.argtypes = [i16p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_Leaf),
                                                  ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                                  ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint8)]
            lib.oracle_detect_removal.restype = ctypes.c_int
            lib.oracle_lines.argtypes = [ctypes.POINTER(_Leaf), ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64)]
            lib.oracle_lines.restype = ctypes.c_int
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


def _leaf_cap(n: int, depth: int, T: int) -> int:
    """Leaf buffer size that lets a detection run once: an upper bound of the
    leaf count.  A line's slope is below 1/2 in cell units, so it crosses at
    most 3 cells of each of the K columns, and every leaf holds at least T
    votes.  Capped at 2^26 leaves (1 GiB of address space; numpy leaves the
    pages untouched until the oracle writes them), beyond which a second run
    sizes the buffer."""
    cap = 1 << 16
    if 1 <= depth <= 24 and T >= 1:
        K = 1 << depth
        cap = max(cap, min(2 * K * K, 2 * (3 * K * n // T + 1), 1 << 26))
    return cap


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
    cap = _leaf_cap(n, depth, T)
    while True:
        leaves = np.empty((cap, 4), dtype=np.uint32)
        rc = lib.oracle_detect(pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), n, W, H, depth, T, m,
                               leaves.ctypes.data_as(ctypes.POINTER(_Leaf)), cap, ctypes.byref(nl),
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
    lv = leaves[:k].copy()
    del leaves
    reg = None
    if dump_regions:
        r = min(int(nr.value), region_cap)
        reg = np.frombuffer(regions, dtype=np.uint32).reshape(-1, 6)[:r].copy()
        if int(nr.value) > region_cap:
            raise RuntimeError("oracle: region dump capacity exceeded")
    return OracleResult(lv, stats, reg, rc)


def sobel(image: np.ndarray, x: int, y: int):
    """(gx, gy) of Sobel's operator at interior pixel (x, y) of a uint8 [H, W] image."""
    img = np.ascontiguousarray(image, dtype=np.uint8)
    H, W = img.shape
    if not (1 <= x <= W - 2 and 1 <= y <= H - 2):
        raise ValueError("oracle.sobel: not an interior pixel")
    gx, gy = ctypes.c_int32(), ctypes.c_int32()
    _load().oracle_sobel(img.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), W, H, x, y, ctypes.byref(gx),
                         ctypes.byref(gy))
    return int(gx.value), int(gy.value)


def edges(image: np.ndarray, threshold: int):
    """Sobel edge points of a uint8 [H, W] image split into ALPHA (|gx| <= |gy|)
    and BETA, each int16 [k, 2] (x, y) in row-major order (Section 3)."""
    img = np.ascontiguousarray(image, dtype=np.uint8)
    H, W = img.shape
    lib = _load()
    cap = max(1, W * H)
    a = np.zeros((cap, 2), np.int16)
    b = np.zeros((cap, 2), np.int16)
    na, nb = ctypes.c_int64(), ctypes.c_int64()
    i16p = ctypes.POINTER(ctypes.c_int16)
    rc = lib.oracle_edges(img.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), W, H, int(threshold),
                          a.ctypes.data_as(i16p), cap, ctypes.byref(na), b.ctypes.data_as(i16p), cap,
                          ctypes.byref(nb))
    if rc != 0:
        raise ValueError(f"oracle.edges failed with code {rc}")
    return a[: na.value].copy(), b[: nb.value].copy()


def detect_split(alpha: np.ndarray, beta: np.ndarray, W: int, H: int, depth: int, T: int) -> OracleResult:
    """Section 3 with the front end's split: ALPHA is processed as given (half
    0) and BETA with x and y swapped (half 1).  That is half 0 of a run on the
    ALPHA points and half 1 of a run on the BETA points; leaves of ALPHA come
    first, as the paper processes ALPHA first."""
    ra = detect(alpha, W, H, depth, T)
    rb = detect(beta, W, H, depth, T)
    la = ra.leaves[ra.leaves[:, 0] == 0] if len(ra.leaves) else ra.leaves
    lb = rb.leaves[rb.leaves[:, 0] == 1] if len(rb.leaves) else rb.leaves
    stats = np.stack([ra.stats[0], rb.stats[1]])
    return OracleResult(np.ascontiguousarray(np.concatenate([la, lb]).reshape(-1, 4)), stats, None, 0)


LINE_DTYPE = np.dtype([("half", np.uint32), ("i", np.uint32), ("j", np.uint32), ("votes", np.uint32),
                       ("cells", np.uint32), ("pad", np.uint32), ("total_votes", np.uint64),
                       ("sum_i2", np.uint64), ("sum_j2", np.uint64)])


def lines(leaves: np.ndarray) -> np.ndarray:
    """Clusters of touching leaves (same half, 8-neighbourhood) -> one line
    each: structured array with the peak cell (half, i, j, votes; ties to the
    earlier leaf), the cluster's cell count and total votes, in the order of
    each cluster's first leaf.  Quadratic: for small leaf sets."""
    lv = np.ascontiguousarray(np.asarray(leaves, dtype=np.uint32).reshape(-1, 4))
    n = lv.shape[0]
    out = np.zeros(max(n, 1), dtype=LINE_DTYPE)
    nl = ctypes.c_int64()
    rc = _load().oracle_lines(lv.ctypes.data_as(ctypes.POINTER(_Leaf)), n, out.ctypes.data, max(n, 1),
                              ctypes.byref(nl))
    if rc != 0:
        raise ValueError(f"oracle.lines failed with code {rc}")
    return out[: nl.value].copy()


def line_parameters(half: int, i: int, j: int, depth: int, L: int):
    """Image line of leaf cell (i, j): its centre (m, b) as exact fractions
    m = (2i + 1 - K) / K and b = 2L (2j + 1 - K) / K; half 0 reads y = m x + b,
    half 1 reads x = m y + b."""
    from fractions import Fraction
    K = 1 << depth
    return Fraction(2 * i + 1 - K, K), Fraction(2 * L * (2 * j + 1 - K), K)


def centroid_parameters(line, depth: int, L: int):
    """A cluster's vote-weighted centre (m, b) as exact fractions:
    m = (S_i / V - K) / K, b = 2L (S_j / V - K) / K."""
    from fractions import Fraction
    K = 1 << depth
    V = int(line["total_votes"])
    return (Fraction(int(line["sum_i2"]), V) - K) / K, 2 * L * (Fraction(int(line["sum_j2"]), V) - K) / K


def detect_subtrees(points: np.ndarray, W: int, H: int, depth: int, T: int, split_level: int,
                    keep: np.ndarray) -> OracleResult:
    """One shard of a detection split by level-`split_level` subtrees: keep is
    uint8 [2 * 4**k] (half, a, b); regions of that level that are not kept are
    tested and counted but not split."""
    lib = _load()
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int16).reshape(-1, 2))
    km = np.ascontiguousarray(np.asarray(keep, dtype=np.uint8).reshape(-1))
    if km.size != 2 * 4 ** split_level:
        raise ValueError("keep must hold 2 * 4**split_level entries")
    stats = np.zeros((2, depth + 1, 4), dtype=np.uint64)
    nl = ctypes.c_int64(0)
    cap = _leaf_cap(pts.shape[0], depth, T)
    while True:
        leaves = np.empty((cap, 4), dtype=np.uint32)
        rc = lib.oracle_detect_subtrees(pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), pts.shape[0], W, H,
                                        depth, T, split_level, km.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                        leaves.ctypes.data_as(ctypes.POINTER(_Leaf)), cap, ctypes.byref(nl),
                                        stats.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        if rc == -4:
            cap = int(nl.value) + 1
            continue
        break
    if rc != 0:
        raise ValueError(f"oracle.detect_subtrees failed with code {rc}")
    lv = leaves[: int(nl.value)].copy()
    return OracleResult(lv, stats, None, rc)


def detect_removal(points: np.ndarray, W: int, H: int, depth: int, T: int):
    """Section 3 with the solution() step: the voters of every accepted leaf
    are plotted and removed from the regions reached later (per half).
    Returns (OracleResult with the accepted leaves in traversal order and the
    statistics, plotted uint8 [2, n])."""
    lib = _load()
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int16).reshape(-1, 2))
    n = pts.shape[0]
    stats = np.zeros((2, depth + 1, 4), dtype=np.uint64)
    plotted = np.zeros((2, max(n, 1)), dtype=np.uint8)
    nl = ctypes.c_int64(0)
    cap = 1 << 14
    while True:
        leaves = (_Leaf * cap)()
        rc = lib.oracle_detect_removal(pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int16)), n, W, H, depth, T,
                                       leaves, cap, ctypes.byref(nl),
                                       stats.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                       plotted.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        if rc == -4:
            cap = int(nl.value) + 1
            continue
        break
    if rc != 0:
        raise ValueError(f"oracle.detect_removal failed with code {rc}")
    lv = np.frombuffer(leaves, dtype=np.uint32).reshape(-1, 4)[: int(nl.value)].copy()
    return OracleResult(lv, stats, None, rc), plotted[:, :n].copy()
