"""C-ABI library checks that need no GPU: it builds, loads, and exports every
function that include/hht.h declares; host-only calls behave as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hht.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hht_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1007_0547_gb300 import build as b
    b.build()
    from paper_1007_0547_gb300 import hht
    return hht.load()


def test_header_declares_the_api():
    assert set(_declared()) == {"hht_create", "hht_destroy", "hht_detect", "hht_detect_batch", "hht_fetch_leaves",
                                "hht_submit", "hht_poll", "hht_progress", "hht_profile_enable", "hht_profile_read",
                                "hht_strerror", "hht_version", "hht_detect_noalloc", "hht_autotune",
                                "hht_set_tuning", "hht_set_batch_mode", "hht_fetch_all_leaves",
                                "hht_inject_fault", "hht_set_predicate", "hht_edges", "hht_detect_image",
                                "hht_lines", "hht_detect_subtrees", "hht_detect_removal",
                                "hht_detect_removal_batch", "hht_create_with_allocator",
                                "hht_done_tickets", "hht_removal_raster"}


def test_library_exports_every_declared_symbol(lib):
    from paper_1007_0547_gb300 import hht
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in hht.EXPORTS


def test_host_only_calls(lib):
    from paper_1007_0547_gb300 import hht
    assert "sm_103a" in hht.version()
    assert hht.strerror(hht.HHT_E_RANGE) == "point outside the image"
    assert hht.strerror(12345) == "unknown error"
    # argument errors are reported before any device work
    assert lib.hht_create(None, 0, None, 0) == hht.HHT_E_ARG
    assert lib.hht_create_with_allocator(None, 0, None, 0, None) == hht.HHT_E_ARG
    h = ctypes.c_void_p()
    assert lib.hht_create_with_allocator(ctypes.byref(h), 0, None, 0, ctypes.byref(hht._Allocator())) == hht.HHT_E_ARG
    r = hht._Result()
    assert lib.hht_detect(None, None, 0, 8, 8, 3, 1, ctypes.byref(r)) == hht.HHT_E_ARG
    assert lib.hht_detect_batch(None, None, 0, None) == hht.HHT_E_ARG
    assert lib.hht_progress(None) == hht.HHT_E_ARG
    assert lib.hht_poll(None, 1, ctypes.byref(r)) == hht.HHT_E_ARG
    assert lib.hht_profile_enable(None, 1) == hht.HHT_E_ARG
    assert lib.hht_profile_read(None, None) == hht.HHT_E_ARG
    assert lib.hht_fetch_leaves(None, 0, None, 0) == hht.HHT_E_ARG
    assert lib.hht_set_tuning(None, 0) == hht.HHT_E_ARG
    assert lib.hht_set_batch_mode(None, 1) == hht.HHT_E_ARG
    assert lib.hht_fetch_all_leaves(None, None, 0, None, None, None) == hht.HHT_E_ARG
    assert lib.hht_autotune(None, None, 0, None, None) == hht.HHT_E_ARG
    assert lib.hht_inject_fault(None, hht.FAULT_WITHHOLD_SCAN_TILE, 0) == hht.HHT_E_ARG
    assert lib.hht_set_predicate(None, hht.PREDICATE_FHT) == hht.HHT_E_ARG
    na, nb = ctypes.c_uint64(), ctypes.c_uint64()
    assert lib.hht_edges(None, None, 8, 8, 10, None, 0, ctypes.byref(na), None, 0, ctypes.byref(nb)) == hht.HHT_E_ARG
    assert lib.hht_detect_image(None, None, 8, 8, 10, 3, 1, ctypes.byref(r)) == hht.HHT_E_ARG
    assert lib.hht_lines(None, 0, None, 0, ctypes.byref(na)) == hht.HHT_E_ARG
    assert lib.hht_removal_raster(None, 0, None, 0) == hht.HHT_E_ARG
    assert lib.hht_detect_subtrees(None, None, 0, 8, 8, 3, 1, 1, None, ctypes.byref(r)) == hht.HHT_E_ARG
    assert lib.hht_detect_removal(None, None, 0, 8, 8, 3, 1, ctypes.byref(r), None) == hht.HHT_E_ARG
    assert lib.hht_detect_removal_batch(None, None, 0, None) == hht.HHT_E_ARG
    assert lib.hht_done_tickets(None, None, 0, ctypes.byref(na)) == hht.HHT_E_ARG


def test_result_struct_layout_matches_header(lib):
    from paper_1007_0547_gb300 import hht
    # leaves, capacity, n_leaves (3 x 8) + depth, L, status, reserved (4 x 4) + stats 2 x 25 x 4 x 8
    assert ctypes.sizeof(hht._Result) == 24 + 16 + 2 * 25 * 4 * 8
    assert ctypes.sizeof(hht._Image) == 8 + 8 + 16


def test_package_fails_loudly_without_library(tmp_path):
    from paper_1007_0547_gb300 import hht
    saved = hht._lib
    try:
        hht._lib = None
        with pytest.raises(ImportError):
            hht.load(str(tmp_path / "missing.so"))
    finally:
        hht._lib = saved


def test_caller_leaf_buffer_is_checked_before_any_call():
    import numpy as np
    import torch
    from paper_1007_0547_gb300 import hht
    buf, ptr, cap = hht.Context._out_buffer(np.zeros((7, 4), np.int32))
    assert cap == 7 and ptr == buf.ctypes.data
    t = torch.zeros((5, 4), dtype=torch.int32)
    assert hht.Context._out_buffer(t)[2] == 5
    for bad in (np.zeros((7, 4), np.int64), np.zeros((7, 3), np.int32), np.zeros((4, 7), np.int32).T,
                torch.zeros((5, 4), dtype=torch.int64), torch.zeros(20, dtype=torch.int32)):
        with pytest.raises(ValueError):
            hht.Context._out_buffer(bad)


def test_binding_structs_match_the_header_as_compiled(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal those a C compiler
    gives the public header's structs."""
    import shutil
    import subprocess
    from paper_1007_0547_gb300 import hht
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"hht_result": hht._Result, "hht_image": hht._Image, "hht_profile_counters": hht._Profile,
               "hht_line": hht._Line}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hht.h"', 'int main(void) {']
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run([cc, "-std=c99", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(w[0], w[1]): int(w[2]) for w in (l.split() for l in out) if len(w) == 3}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
