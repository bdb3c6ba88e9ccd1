"""Python binding of libhht.so (ctypes): argument marshalling only.

Every step of the detection runs in the library's CUDA kernels; PyTorch is
used here for device memory and the CUDA stream.  Importing this module
builds nothing and falls back to nothing: when the compiled library is absent
the import fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import sys
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhht.so")
MAX_DEPTH = 24

HHT_OK = 0
HHT_E_ARG = -1
HHT_E_RANGE = -2
HHT_E_CAPACITY = -3
HHT_E_NOMEM = -4
HHT_E_TIMEOUT = -5
HHT_E_CUDA = -6
HHT_E_PENDING = -7
HHT_E_UNKNOWN_TICKET = -8

# every function the C header declares
EXPORTS = ("hht_create", "hht_destroy", "hht_detect", "hht_detect_batch", "hht_fetch_leaves", "hht_submit",
           "hht_poll", "hht_progress", "hht_profile_enable", "hht_profile_read", "hht_strerror", "hht_version",
           "hht_detect_noalloc", "hht_autotune", "hht_set_tuning", "hht_set_batch_mode", "hht_fetch_all_leaves",
           "hht_inject_fault", "hht_set_predicate", "hht_edges", "hht_detect_image", "hht_lines",
           "hht_detect_subtrees", "hht_detect_removal", "hht_detect_removal_batch",
           "hht_create_with_allocator", "hht_done_tickets", "hht_removal_raster")
BATCH_LEVELS, BATCH_GRAPH = 0, 1
BATCH_PERSISTENT = BATCH_GRAPH  # earlier name
FAULT_NONE, FAULT_WITHHOLD_SCAN_TILE, FAULT_GRAPH_CAPACITY = 0, 1, 2
PREDICATE_EXACT, PREDICATE_FHT = 0, 1
TUNE_SHAPES = 6


class HhtError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


class _Result(ctypes.Structure):
    _fields_ = [("leaves", ctypes.c_void_p), ("leaf_capacity", ctypes.c_uint64), ("n_leaves", ctypes.c_uint64),
                ("depth", ctypes.c_int32), ("L", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("stats", ctypes.c_uint64 * (2 * (MAX_DEPTH + 1) * 4))]


class _Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("pass_launches", ctypes.c_uint64),
                ("select_launches", ctypes.c_uint64), ("voters_read", ctypes.c_uint64),
                ("voters_written", ctypes.c_uint64), ("pass_bytes", ctypes.c_uint64), ("pass_ms", ctypes.c_double),
                ("select_ms", ctypes.c_double), ("stage_ms", ctypes.c_double),
                ("graph_launches", ctypes.c_uint64), ("graph_fallbacks", ctypes.c_uint64),
                ("edges_launches", ctypes.c_uint64), ("edges_pixels", ctypes.c_uint64),
                ("edges_points", ctypes.c_uint64), ("edges_ms", ctypes.c_double),
                ("graph_captures", ctypes.c_uint64)]


class _Line(ctypes.Structure):
    _fields_ = [("half", ctypes.c_uint32), ("i", ctypes.c_uint32), ("j", ctypes.c_uint32), ("votes", ctypes.c_uint32),
                ("cells", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("total_votes", ctypes.c_uint64),
                ("sum_i2", ctypes.c_uint64), ("sum_j2", ctypes.c_uint64)]


LINE_DTYPE = np.dtype([("half", np.uint32), ("i", np.uint32), ("j", np.uint32), ("votes", np.uint32),
                       ("cells", np.uint32), ("reserved", np.uint32), ("total_votes", np.uint64),
                       ("sum_i2", np.uint64), ("sum_j2", np.uint64)])


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


def _torch_allocator(device: int) -> _Allocator:
    """The library's scratch memory from PyTorch's caching allocator (on the
    context's stream), so that it shows up in torch's memory statistics and
    its blocks return to torch's cache when the context frees them."""
    import torch

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:  # out of memory: the library reports HHT_E_NOMEM
            return None

    def free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    return _Allocator(_ALLOC_FN(alloc), _FREE_FN(free), None)


class _Image(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("n", ctypes.c_int64), ("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("T", ctypes.c_int32)]


_lib = None


def load(path: Optional[str] = None):
    """Load libhht.so (the in-tree build, or the file $HHT_LIB names); raises
    if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("HHT_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1007_0547_gb300.build` "
                          "(needs nvcc); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    lib.hht_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, u64]
    lib.hht_create.restype = ctypes.c_int
    lib.hht_create_with_allocator.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, u64, ctypes.POINTER(_Allocator)]
    lib.hht_create_with_allocator.restype = ctypes.c_int
    lib.hht_destroy.argtypes = [vp]
    lib.hht_destroy.restype = None
    lib.hht_detect.argtypes = [vp, vp, i64, i32, i32, i32, i32, ctypes.POINTER(_Result)]
    lib.hht_detect.restype = ctypes.c_int
    lib.hht_detect_batch.argtypes = [vp, ctypes.POINTER(_Image), i32, ctypes.POINTER(_Result)]
    lib.hht_detect_batch.restype = ctypes.c_int
    lib.hht_fetch_all_leaves.argtypes = [vp, vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.hht_fetch_all_leaves.restype = ctypes.c_int
    lib.hht_fetch_leaves.argtypes = [vp, i32, vp, u64]
    lib.hht_fetch_leaves.restype = ctypes.c_int
    lib.hht_submit.argtypes = [vp, ctypes.POINTER(_Image), ctypes.POINTER(u64)]
    lib.hht_submit.restype = ctypes.c_int
    lib.hht_poll.argtypes = [vp, u64, ctypes.POINTER(_Result)]
    lib.hht_poll.restype = ctypes.c_int
    lib.hht_progress.argtypes = [vp]
    lib.hht_progress.restype = ctypes.c_int
    lib.hht_done_tickets.argtypes = [vp, ctypes.POINTER(u64), u64, ctypes.POINTER(u64)]
    lib.hht_done_tickets.restype = ctypes.c_int
    lib.hht_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.hht_profile_enable.restype = ctypes.c_int
    lib.hht_profile_read.argtypes = [vp, ctypes.POINTER(_Profile)]
    lib.hht_profile_read.restype = ctypes.c_int
    lib.hht_autotune.argtypes = [vp, ctypes.POINTER(_Image), i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
    lib.hht_autotune.restype = ctypes.c_int
    lib.hht_set_batch_mode.argtypes = [vp, i32]
    lib.hht_set_batch_mode.restype = ctypes.c_int
    lib.hht_set_tuning.argtypes = [vp, i32]
    lib.hht_set_tuning.restype = ctypes.c_int
    lib.hht_inject_fault.argtypes = [vp, i32, i64]
    lib.hht_inject_fault.restype = ctypes.c_int
    lib.hht_set_predicate.argtypes = [vp, i32]
    lib.hht_set_predicate.restype = ctypes.c_int
    lib.hht_detect_removal.argtypes = [vp, vp, i64, i32, i32, i32, i32, ctypes.POINTER(_Result), vp]
    lib.hht_detect_removal.restype = ctypes.c_int
    lib.hht_detect_removal_batch.argtypes = [vp, ctypes.POINTER(_Image), i32, ctypes.POINTER(_Result)]
    lib.hht_detect_removal_batch.restype = ctypes.c_int
    lib.hht_removal_raster.argtypes = [vp, i32, vp, u64]
    lib.hht_removal_raster.restype = ctypes.c_int
    lib.hht_detect_subtrees.argtypes = [vp, vp, i64, i32, i32, i32, i32, i32, vp, ctypes.POINTER(_Result)]
    lib.hht_detect_subtrees.restype = ctypes.c_int
    lib.hht_lines.argtypes = [vp, i32, vp, u64, ctypes.POINTER(u64)]
    lib.hht_lines.restype = ctypes.c_int
    lib.hht_edges.argtypes = [vp, vp, i32, i32, i32, vp, u64, ctypes.POINTER(u64), vp, u64, ctypes.POINTER(u64)]
    lib.hht_edges.restype = ctypes.c_int
    lib.hht_detect_image.argtypes = [vp, vp, i32, i32, i32, i32, i32, ctypes.POINTER(_Result)]
    lib.hht_detect_image.restype = ctypes.c_int
    lib.hht_strerror.argtypes = [ctypes.c_int]
    lib.hht_strerror.restype = ctypes.c_char_p
    lib.hht_version.argtypes = []
    lib.hht_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().hht_strerror(int(code)).decode()
    except ImportError:
        return f"error {code}"


@dataclasses.dataclass
class Result:
    leaves: "object"      # [k, 4] int32 (half, i, j, votes): torch tensor (device) or numpy (host)
    stats: np.ndarray     # uint64 [2, depth + 1, 4]: tested, passed, votes, tests
    depth: int
    L: int
    status: int

    @property
    def n_leaves(self) -> int:
        return int(self.leaves.shape[0])

    def total_tests(self) -> int:
        return int(self.stats[:, :, 3].sum())

    def leaves_numpy(self) -> np.ndarray:
        lv = self.leaves
        if hasattr(lv, "detach"):
            lv = lv.detach().cpu().numpy()
        return np.asarray(lv).astype(np.uint32).reshape(-1, 4)


# numpy view of an array of _Result (fields at the ctypes offsets)
_RESULT_DTYPE = np.dtype({
    "names": [f for f, _ in _Result._fields_],
    "formats": [np.uint64, np.uint64, np.uint64, np.int32, np.int32, np.int32, np.int32,
                (np.uint64, (2 * (MAX_DEPTH + 1) * 4,))],
    "offsets": [getattr(_Result, f).offset for f, _ in _Result._fields_],
    "itemsize": ctypes.sizeof(_Result)})


# A status the library never writes: marks the results of images that a batch
# call returned without reaching.
_NOT_REACHED = 1


def _stats_of(r: _Result) -> np.ndarray:
    st = np.frombuffer(r.stats, dtype=np.uint64).reshape(2, MAX_DEPTH + 1, 4)
    return st[:, : r.depth + 1].copy()


class _Points:
    """Keeps a contiguous int16 [n, 2] buffer alive and exposes its address."""

    def __init__(self, points):
        self.keep = None
        try:
            import torch
            if isinstance(points, torch.Tensor):
                t = points
                if t.dtype != torch.int16 or t.dim() != 2 or t.shape[1] != 2 or not t.is_contiguous():
                    t = t.to(torch.int16).contiguous().reshape(-1, 2)
                self.keep = t
                self.ptr = t.data_ptr() if t.numel() else None
                self.n = t.shape[0]
                self.device = t.is_cuda
                return
        except ImportError:  # pragma: no cover
            pass
        a = np.ascontiguousarray(np.asarray(points, dtype=np.int16).reshape(-1, 2))
        self.keep = a
        self.ptr = a.ctypes.data if a.size else None
        self.n = a.shape[0]
        self.device = False


class Context:
    """One library context: device, CUDA stream (the current torch stream at
    creation unless given) and the scratch memory it holds."""

    def __init__(self, device: int = 0, stream=None, mem_budget: int = 0, allocator: Optional[str] = None):
        """allocator: None (the library's cudaMalloc) or "torch" (PyTorch's
        caching allocator holds the context's scratch memory)."""
        import torch
        lib = load()
        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        handle = ctypes.c_void_p()
        sp = ctypes.c_void_p(int(stream.cuda_stream)) if hasattr(stream, "cuda_stream") else ctypes.c_void_p(stream)
        if allocator not in (None, "torch"):
            raise ValueError('allocator must be None or "torch"')
        self._allocator = _torch_allocator(self.device) if allocator == "torch" else None
        if self._allocator is not None:
            rc = lib.hht_create_with_allocator(ctypes.byref(handle), self.device, sp, int(mem_budget),
                                               ctypes.byref(self._allocator))
        else:
            rc = lib.hht_create(ctypes.byref(handle), self.device, sp, int(mem_budget))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_create")
        self._h = handle
        self._cap_hint = 1 << 12

    def close(self):
        if getattr(self, "_h", None):
            load().hht_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        # At interpreter exit PyTorch may already be torn down: a context whose
        # memory comes from torch's allocator is then left to the process exit
        # instead of calling back into torch.
        if sys.is_finalizing() and getattr(self, "_allocator", None) is not None:
            return
        try:
            self.close()
        except Exception:
            pass

    def _alloc_leaves(self, cap: int, on_device: bool, pinned: bool = False):
        import torch
        if on_device:
            buf = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=f"cuda:{self.device}")
            return buf, buf.data_ptr()
        if pinned and cap > 0:
            # page-locked memory from PyTorch's caching host allocator (reused
            # across calls): the device -> host copy runs at link speed instead
            # of through the driver's staging of pageable memory; the numpy
            # view keeps the tensor alive
            t = torch.empty((cap, 4), dtype=torch.int32, pin_memory=True)
            return t.numpy(), t.data_ptr()
        buf = np.empty((max(cap, 1), 4), dtype=np.int32)
        return buf, buf.ctypes.data

    @staticmethod
    def _out_buffer(out):
        """A caller's leaf buffer: int32 [cap, 4] (numpy array or torch tensor,
        host or device, contiguous) -> (buffer, address, capacity)."""
        try:
            import torch
            if isinstance(out, torch.Tensor):
                if out.dtype != torch.int32 or out.dim() != 2 or out.shape[1] != 4 or not out.is_contiguous():
                    raise ValueError("leaves_out must be a contiguous int32 tensor of shape [capacity, 4]")
                return out, out.data_ptr(), int(out.shape[0])
        except ImportError:  # pragma: no cover
            pass
        if not (isinstance(out, np.ndarray) and out.dtype == np.int32 and out.ndim == 2 and out.shape[1] == 4
                and out.flags.c_contiguous):
            raise ValueError("leaves_out must be a C-contiguous int32 array of shape [capacity, 4]")
        return out, out.ctypes.data, int(out.shape[0])

    def _fetch(self, index: int, n: int, on_device: bool):
        """Leaves of image `index` of the last job (no recomputation)."""
        buf, ptr = self._alloc_leaves(n, on_device)
        rc = load().hht_fetch_leaves(self._h, int(index), ptr, n)
        if rc != HHT_OK:
            raise HhtError(rc, "hht_fetch_leaves")
        return buf

    def detect(self, points, W: int, H: int, depth: int, T: int, leaves_on_device: bool = True,
               leaf_capacity: Optional[int] = None, raise_on_error: bool = True, leaves_out=None) -> Result:
        """Detect one image.  The leaves land in a new buffer (on the device
        unless leaves_on_device is False) or, with `leaves_out` (an int32
        [capacity, 4] host or device buffer, e.g. pinned host memory reused
        across calls), in that buffer: the result's leaves are then a view of it."""
        lib = load()
        p = _Points(points)
        if leaves_out is not None:
            buf, ptr, cap = self._out_buffer(leaves_out)
        else:
            cap = int(leaf_capacity or self._cap_hint)
            buf, ptr = self._alloc_leaves(cap, leaves_on_device)
        r = _Result()
        r.leaves = ptr
        r.leaf_capacity = cap
        rc = lib.hht_detect(self._h, p.ptr, p.n, int(W), int(H), int(depth), int(T), ctypes.byref(r))
        if rc == HHT_E_CAPACITY:
            if leaves_out is not None:
                raise ValueError(f"leaves_out holds {cap} leaves, the image has {int(r.n_leaves)}")
            # the leaves are kept by the context: copy them into a buffer of the right size
            self._cap_hint = max(self._cap_hint, int(r.n_leaves))
            buf = self._fetch(0, int(r.n_leaves), leaves_on_device)
            rc = HHT_OK
        if rc != HHT_OK and raise_on_error:
            raise HhtError(rc, "hht_detect")
        k = int(r.n_leaves) if rc == HHT_OK else 0
        return Result(buf[:k], _stats_of(r), int(r.depth), int(r.L), rc)

    def detect_batch(self, images: Sequence[Tuple], leaves_on_device: bool = True,
                     raise_on_error: bool = True, leaves_out=None) -> List[Result]:
        """images: sequence of (points, W, H, depth, T).  The leaves of all
        images land in one new buffer (on the device unless leaves_on_device
        is False) or in `leaves_out` (an int32 [capacity, 4] host or device
        buffer, e.g. pinned host memory reused across calls); each result's
        leaves are a view of that buffer."""
        lib = load()
        nimg = len(images)
        if nimg == 0:
            return []
        pts = [_Points(im[0]) for im in images]
        arr = (_Image * nimg)()
        for k, (im, p) in enumerate(zip(images, pts)):
            arr[k].points = p.ptr
            arr[k].n = p.n
            arr[k].W, arr[k].H, arr[k].depth, arr[k].T = (int(v) for v in im[1:5])
        # no leaves are copied by the batch call itself: all leaves of the job
        # are fetched afterwards with one copy, and each image gets a view
        outs = (_Result * nimg)()
        np.frombuffer(outs, dtype=_RESULT_DTYPE)["status"] = _NOT_REACHED
        rc = lib.hht_detect_batch(self._h, arr, nimg, outs)
        if (np.frombuffer(outs, dtype=_RESULT_DTYPE)["status"] == _NOT_REACHED).any():
            # the call returned before reporting every image (an argument error,
            # or a wave that failed as a whole): the context holds no complete
            # job of these images, so nothing is fetched
            code = rc if rc != HHT_OK else HHT_E_CUDA
            if raise_on_error:
                raise HhtError(code, "hht_detect_batch")
            empty = self._alloc_leaves(0, leaves_on_device)[0][:0]
            return [Result(empty, np.zeros((2, int(im[3]) + 1, 4), np.uint64), int(im[3]), 0, code)
                    for im in images]
        for k in range(nimg):
            if outs[k].status == HHT_E_CAPACITY:
                outs[k].status = HHT_OK
        if rc == HHT_E_CAPACITY:
            rc = HHT_OK
        total = ctypes.c_uint64()
        offs = (ctypes.c_uint64 * nimg)()
        cnts = (ctypes.c_uint64 * nimg)()
        lib.hht_fetch_all_leaves(self._h, None, 0, offs, cnts, ctypes.byref(total))
        if leaves_out is not None:
            allbuf, ptr, cap = self._out_buffer(leaves_out)
            if cap < int(total.value):
                raise ValueError(f"leaves_out holds {cap} leaves, the batch has {int(total.value)}")
        else:
            allbuf, ptr = self._alloc_leaves(int(total.value), leaves_on_device)
        frc = lib.hht_fetch_all_leaves(self._h, ptr, int(total.value), offs, cnts, ctypes.byref(total))
        if frc != HHT_OK:
            raise HhtError(frc, "hht_fetch_all_leaves")
        # per-image views and statistics from one numpy view of the result array
        o = np.frombuffer(offs, dtype=np.uint64).astype(np.int64)
        rows = np.frombuffer(outs, dtype=_RESULT_DTYPE)
        n_leaves = rows["n_leaves"].astype(np.int64)
        status = rows["status"].astype(np.int64)
        depth = rows["depth"].astype(np.int64)
        Ls = rows["L"].astype(np.int64)
        stats = rows["stats"].reshape(nimg, 2, MAX_DEPTH + 1, 4)
        res = []
        for k in range(nimg):
            st = int(status[k])
            if st != HHT_OK and raise_on_error:
                raise HhtError(st, f"hht_detect_batch[{k}]")
            nk = int(n_leaves[k]) if st == HHT_OK else 0
            dk = int(depth[k])
            res.append(Result(allbuf[int(o[k]): int(o[k]) + nk], stats[k, :, : dk + 1].copy(), dk, int(Ls[k]), st))
        if rc != HHT_OK and raise_on_error:
            raise HhtError(rc, "hht_detect_batch")
        return res

    def set_batch_mode(self, mode: int) -> None:
        """BATCH_GRAPH (default: the device-driven level loop, one CUDA-graph
        launch and one host synchronisation per job, buffers sized from upper
        bounds) or BATCH_LEVELS (one selection and one level-kernel launch per
        level with a host synchronisation each, buffers sized exactly)."""
        rc = load().hht_set_batch_mode(self._h, int(mode))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_set_batch_mode")

    # ------------------------------------------------------------ autotuning
    def set_tuning(self, shape: int) -> None:
        rc = load().hht_set_tuning(self._h, int(shape))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_set_tuning")

    def autotune(self, images: Sequence[Tuple], cache: Optional[str] = None) -> Tuple[int, Optional[List[float]]]:
        """Pick the level kernel's tile shape for workloads like `images`
        ((points, W, H, depth, T) tuples).  With `cache` (a JSON file, default
        $HHT_TUNE_CACHE), the choice is stored per (device, workload class) and
        reused without timing."""
        import json
        import math
        import torch
        cache = cache or os.environ.get("HHT_TUNE_CACHE")
        n_total = sum(_Points(im[0]).n for im in images)
        key = (f"{torch.cuda.get_device_name(self.device)}|{load().hht_version().decode()}|images={len(images)}|"
               f"points~2^{int(math.log2(max(1, n_total)))}|depth<={max(int(im[3]) for im in images)}")
        table = {}
        if cache and os.path.exists(cache):
            try:
                with open(cache) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
        if key in table:
            self.set_tuning(int(table[key]["shape"]))
            return int(table[key]["shape"]), None
        pts = [_Points(im[0]) for im in images]
        arr = (_Image * len(images))()
        for k, (im, p) in enumerate(zip(images, pts)):
            arr[k].points = p.ptr
            arr[k].n = p.n
            arr[k].W, arr[k].H, arr[k].depth, arr[k].T = (int(v) for v in im[1:5])
        best = ctypes.c_int32()
        ms = (ctypes.c_double * TUNE_SHAPES)()
        rc = load().hht_autotune(self._h, arr, len(images), ctypes.byref(best), ms)
        if rc != HHT_OK:
            raise HhtError(rc, "hht_autotune")
        times = [float(v) for v in ms]
        if cache:
            table[key] = {"shape": int(best.value), "pass_ms": times}
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1)
            os.replace(tmp, cache)
        return int(best.value), times

    # ------------------------------------------------------------ kernel timing
    @staticmethod
    def _image(image):
        """A grey-level image (uint8 [H, W], numpy or torch, host or device) ->
        (keep-alive, address, W, H)."""
        try:
            import torch
            if isinstance(image, torch.Tensor):
                if image.dtype != torch.uint8 or image.dim() != 2:
                    raise ValueError("image must be a uint8 tensor of shape [H, W]")
                t = image.contiguous()
                return t, t.data_ptr(), int(t.shape[1]), int(t.shape[0])
        except ImportError:  # pragma: no cover
            pass
        a = np.ascontiguousarray(image)
        if a.dtype != np.uint8 or a.ndim != 2:
            raise ValueError("image must be a uint8 array of shape [H, W]")
        return a, a.ctypes.data, int(a.shape[1]), int(a.shape[0])

    def edges(self, image, threshold: int, on_device: bool = True):
        """Sobel edge points of a grey-level image split into ALPHA and BETA
        (Section 3): two int16 [k, 2] (x, y) buffers, row-major order each."""
        import torch
        lib = load()
        keep, ptr, W, H = self._image(image)
        # one call with buffers that hold every interior pixel (the most either list can get)
        cap = max(1, (W - 2) * (H - 2)) if W >= 3 and H >= 3 else 1
        dev = f"cuda:{self.device}" if on_device else "cpu"
        a = torch.empty((cap, 2), dtype=torch.int16, device=dev)
        b = torch.empty((cap, 2), dtype=torch.int16, device=dev)
        na, nb = ctypes.c_uint64(), ctypes.c_uint64()
        rc = lib.hht_edges(self._h, ptr, W, H, int(threshold), a.data_ptr(), cap, ctypes.byref(na),
                           b.data_ptr(), cap, ctypes.byref(nb))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_edges")
        del keep
        return a[: int(na.value)], b[: int(nb.value)]

    def detect_image(self, image, threshold: int, depth: int, T: int, leaves_on_device: bool = True,
                     raise_on_error: bool = True) -> Result:
        """Front end plus detection: Sobel edges split into ALPHA (half 0) and
        BETA (half 1, x and y swapped), then the hierarchy on each."""
        lib = load()
        keep, ptr, W, H = self._image(image)
        cap = int(self._cap_hint)
        buf, lp = self._alloc_leaves(cap, leaves_on_device)
        r = _Result()
        r.leaves = lp
        r.leaf_capacity = cap
        rc = lib.hht_detect_image(self._h, ptr, W, H, int(threshold), int(depth), int(T), ctypes.byref(r))
        if rc == HHT_E_CAPACITY:
            self._cap_hint = max(self._cap_hint, int(r.n_leaves))
            buf = self._fetch(0, int(r.n_leaves), leaves_on_device)
            rc = HHT_OK
        if rc != HHT_OK and raise_on_error:
            raise HhtError(rc, "hht_detect_image")
        del keep
        k = int(r.n_leaves) if rc == HHT_OK else 0
        return Result(buf[:k], _stats_of(r), int(r.depth), int(r.L), rc)

    def detect_removal(self, points, W: int, H: int, depth: int, T: int, with_plotted: bool = True):
        """Detection with the solution() step (hht_detect_removal): accepted
        cells in visiting order and, with with_plotted, uint8 [2, n] flags of
        the plotted points per half.  Returns (Result, plotted or None)."""
        lib = load()
        p = _Points(points)
        cap = max(1, 2 * (p.n // max(int(T), 1) + 1))
        buf = np.zeros((cap, 4), dtype=np.int32)
        plotted = np.zeros((2, max(p.n, 1)), dtype=np.uint8) if with_plotted else None
        r = _Result()
        r.leaves = buf.ctypes.data
        r.leaf_capacity = cap
        rc = lib.hht_detect_removal(self._h, p.ptr, p.n, int(W), int(H), int(depth), int(T), ctypes.byref(r),
                                    plotted.ctypes.data if with_plotted else None)
        if rc != HHT_OK:
            raise HhtError(rc, "hht_detect_removal")
        k = int(r.n_leaves)
        return Result(buf[:k], _stats_of(r), int(r.depth), int(r.L), rc), (plotted[:, : p.n] if with_plotted else None)

    def removal_raster(self, index: int, W: int, H: int, on_device: bool = False):
        """The points that solution() plotted for image `index` of the last
        removal job as a uint8 [H, W] raster (bit 0: half 0, bit 1: half 1),
        numpy on the host or a torch tensor on the device."""
        if on_device:
            import torch
            buf = torch.empty((int(H), int(W)), dtype=torch.uint8, device=f"cuda:{self.device}")
            ptr = buf.data_ptr()
        else:
            buf = np.empty((int(H), int(W)), dtype=np.uint8)
            ptr = buf.ctypes.data
        rc = load().hht_removal_raster(self._h, int(index), ptr, int(W) * int(H))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_removal_raster")
        return buf

    def detect_removal_batch(self, images: Sequence[Tuple]) -> List[Result]:
        """hht_detect_removal_batch over (points, W, H, depth, T) tuples."""
        lib = load()
        pts = [_Points(im[0]) for im in images]
        arr = (_Image * len(images))()
        outs = (_Result * len(images))()
        bufs = []
        for k, (im, p) in enumerate(zip(images, pts)):
            arr[k].points = p.ptr
            arr[k].n = p.n
            arr[k].W, arr[k].H, arr[k].depth, arr[k].T = (int(v) for v in im[1:5])
            cap = max(1, 2 * (p.n // max(int(im[4]), 1) + 1))
            b = np.zeros((cap, 4), dtype=np.int32)
            bufs.append(b)
            outs[k].leaves = b.ctypes.data
            outs[k].leaf_capacity = cap
        rc = lib.hht_detect_removal_batch(self._h, arr, len(images), outs)
        if rc != HHT_OK:
            raise HhtError(rc, "hht_detect_removal_batch")
        return [Result(b[: int(o.n_leaves)], _stats_of(o), int(o.depth), int(o.L), int(o.status))
                for b, o in zip(bufs, outs)]

    def detect_subtrees(self, points, W: int, H: int, depth: int, T: int, split_level: int, keep,
                        leaves_on_device: bool = True) -> Result:
        """One shard of a detection split by level-`split_level` subtrees
        (hht_detect_subtrees): keep is a uint8 mask of 2 * 4**split_level
        entries (half, a, b); see shard.plan_subtrees / merge_subtrees."""
        lib = load()
        p = _Points(points)
        km = np.ascontiguousarray(np.asarray(keep, dtype=np.uint8).reshape(-1))
        if km.size != 2 * 4 ** int(split_level):
            raise ValueError("keep must hold 2 * 4**split_level entries")
        cap = int(self._cap_hint)
        buf, lp = self._alloc_leaves(cap, leaves_on_device)
        r = _Result()
        r.leaves = lp
        r.leaf_capacity = cap
        rc = lib.hht_detect_subtrees(self._h, p.ptr, p.n, int(W), int(H), int(depth), int(T), int(split_level),
                                     km.ctypes.data, ctypes.byref(r))
        if rc == HHT_E_CAPACITY:
            self._cap_hint = max(self._cap_hint, int(r.n_leaves))
            buf = self._fetch(0, int(r.n_leaves), leaves_on_device)
            rc = HHT_OK
        if rc != HHT_OK:
            raise HhtError(rc, "hht_detect_subtrees")
        k = int(r.n_leaves)
        return Result(buf[:k], _stats_of(r), int(r.depth), int(r.L), rc)

    def lines(self, index: int = 0) -> np.ndarray:
        """Lines of image `index` of the last job (hht_lines): a structured
        numpy array (LINE_DTYPE) with each cluster's peak leaf, cell count,
        total votes and the sums of its vote-weighted centre."""
        lib = load()
        n = ctypes.c_uint64()
        rc = lib.hht_lines(self._h, int(index), None, 0, ctypes.byref(n))
        if rc not in (HHT_OK, HHT_E_CAPACITY):
            raise HhtError(rc, "hht_lines")
        out = np.zeros(max(int(n.value), 1), dtype=LINE_DTYPE)
        rc = lib.hht_lines(self._h, int(index), out.ctypes.data, len(out), ctypes.byref(n))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_lines")
        return out[: int(n.value)]

    def set_predicate(self, predicate: int) -> None:
        """PREDICATE_EXACT (the paper's 4-bit code) or PREDICATE_FHT (the
        prior-art circumscribed-circle test) for detect and detect_batch."""
        rc = load().hht_set_predicate(self._h, int(predicate))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_set_predicate")

    def inject_fault(self, kind: int, arg: int = 0) -> None:
        """Host-side fault injection for tests (hht_inject_fault): with
        FAULT_WITHHOLD_SCAN_TILE, tile `arg` of the next job's look-back
        scans publishes nothing, so that job fails with HHT_E_TIMEOUT once the
        bounded waits behind it expire."""
        rc = load().hht_inject_fault(self._h, int(kind), int(arg))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_inject_fault")

    def profile(self, on: bool = True) -> None:
        rc = load().hht_profile_enable(self._h, 1 if on else 0)
        if rc != HHT_OK:
            raise HhtError(rc, "hht_profile_enable")

    def profile_read(self) -> dict:
        p = _Profile()
        rc = load().hht_profile_read(self._h, ctypes.byref(p))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_profile_read")
        return {name: getattr(p, name) for name, _ in _Profile._fields_}

    # ------------------------------------------------------------ serving
    def submit(self, points, W: int, H: int, depth: int, T: int) -> int:
        lib = load()
        p = _Points(points)
        im = _Image(p.ptr, p.n, int(W), int(H), int(depth), int(T))
        t = ctypes.c_uint64()
        rc = lib.hht_submit(self._h, ctypes.byref(im), ctypes.byref(t))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_submit")
        return int(t.value)

    def progress(self) -> int:
        rc = load().hht_progress(self._h)
        if rc < 0:
            raise HhtError(rc, "hht_progress")
        return rc

    def done_tickets(self, max_count: int = 4096) -> List[int]:
        """Tickets of finished requests not polled or listed before
        (hht_done_tickets), oldest completion first."""
        buf = (ctypes.c_uint64 * max_count)()
        n = ctypes.c_uint64()
        rc = load().hht_done_tickets(self._h, buf, max_count, ctypes.byref(n))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_done_tickets")
        return list(buf[: int(n.value)])

    def poll(self, ticket: int, leaves_on_device: bool = False) -> Optional[Result]:
        """None while the request is pending; else its Result (the ticket is
        then released).  A pending poll allocates nothing: the first call asks
        with an empty buffer, and only a finished request gets one of its size."""
        lib = load()
        r = _Result()
        r.leaves = None
        r.leaf_capacity = 0
        rc = lib.hht_poll(self._h, int(ticket), ctypes.byref(r))
        if rc == HHT_E_PENDING:
            return None
        buf, ptr = self._alloc_leaves(0, leaves_on_device)
        while rc == HHT_E_CAPACITY:
            cap = int(r.n_leaves)
            buf, ptr = self._alloc_leaves(cap, leaves_on_device, pinned=True)
            r = _Result()
            r.leaves = ptr
            r.leaf_capacity = cap
            rc = lib.hht_poll(self._h, int(ticket), ctypes.byref(r))
        if rc != HHT_OK:
            raise HhtError(rc, "hht_poll")
        return Result(buf[: int(r.n_leaves)], _stats_of(r), int(r.depth), int(r.L), rc)


_default: Optional[Context] = None


def default_context() -> Context:
    global _default
    if _default is None:
        _default = Context()
    return _default


def detect(points, W: int, H: int, depth: int, T: int, **kw) -> Result:
    """Detect lines in one image with the default context (cuda:0)."""
    return default_context().detect(points, W, H, depth, T, **kw)


def version() -> str:
    return load().hht_version().decode()
