"""C-ABI boundary checks that need no GPU: the library loads, exports every
function include/wg.h declares, and rejects bad arguments before touching the
device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build_library()
    from paper_1203_5004_gb300 import _lib
    return _lib.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "wg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(wg_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_core_api():
    names = declared_functions()
    for must in ("wg_upper_hood", "wg_upper_hood_batched", "wg_upper_hood_workspace_size",
                 "wg_upper_hood_batched_workspace_size", "wg_get_device_status", "wg_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1203_5004_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_binding_declares_nothing_extra():
    from paper_1203_5004_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_status_strings(lib):
    for code in range(8):
        assert lib.wg_status_string(code)


def test_options_default(lib):
    from paper_1203_5004_gb300 import _lib
    o = _lib.default_options()
    assert (o.pred_mode, o.count_predicates, o.validate, o.tile_config, o.segments_per_cta) == (0, 0, 0, 0, 0)


def test_workspace_queries(lib):
    assert lib.wg_upper_hood_workspace_size(0) >= 256
    assert lib.wg_upper_hood_workspace_size(1 << 26) == lib.wg_upper_hood_workspace_size(10)
    # the plain schedule keeps two copies of the hoods: at least 24 bytes per point
    assert lib.wg_upper_hood_plain_workspace_size(1 << 20) >= 24 * (1 << 20)
    off = np.array([0, 5, 5, 70000], dtype=np.int64)
    assert lib.wg_upper_hood_batched_workspace_size(off.ctypes.data, 3) >= 256
    assert lib.wg_upper_hood_batched_workspace_size(None, 0) >= 256
    # the sort keeps two key copies (8 bytes each), an index copy and the histograms
    assert lib.wg_sort_points_workspace_size(1 << 20) >= 20 * (1 << 20)
    assert lib.wg_upper_hood_unsorted_workspace_size(1 << 20) >= \
        lib.wg_upper_hood_workspace_size(1 << 20) + 12 * (1 << 20) + lib.wg_sort_points_workspace_size(1 << 20)


def test_argument_errors_without_device(lib):
    # These fail the argument checks, which run before any CUDA call.
    buf = ctypes.create_string_buffer(1 << 16)
    addr = (ctypes.addressof(buf) + 255) // 256 * 256
    ws_bytes = lib.wg_upper_hood_workspace_size(100)
    # negative n
    assert lib.wg_upper_hood(addr, -1, addr, addr, addr, ws_bytes, None) == 1
    # null outputs
    assert lib.wg_upper_hood(addr, 10, None, addr, addr, ws_bytes, None) == 1
    assert lib.wg_upper_hood(addr, 10, addr, None, addr, ws_bytes, None) == 1
    # misaligned points (4 bytes)
    assert lib.wg_upper_hood(addr + 4, 10, addr, addr, addr, ws_bytes, None) == 1
    # workspace too small / missing
    assert lib.wg_upper_hood(addr, 10, addr, addr, addr, 16, None) == 2
    assert lib.wg_upper_hood(addr, 10, addr, addr, None, ws_bytes, None) == 2
    # n beyond int32
    assert lib.wg_upper_hood(addr, 1 << 31, addr, addr, addr, ws_bytes, None) == 7
    # bad options
    from paper_1203_5004_gb300 import _lib
    o = _lib.default_options(pred_mode=5)
    assert lib.wg_upper_hood_ex(addr, 10, addr, addr, addr, ws_bytes, ctypes.byref(o), None) == 1
    o = _lib.default_options(tile_config=9)
    assert lib.wg_upper_hood_ex(addr, 10, addr, addr, addr, ws_bytes, ctypes.byref(o), None) == 1
    # batched
    assert lib.wg_upper_hood_batched(addr, addr, -1, addr, addr, addr, ws_bytes, None, None) == 1
    # the small-set schedule beyond its size, an unknown schedule
    o = _lib.default_options(schedule=4)
    assert lib.wg_upper_hood_ex(addr, 8193, addr, addr, addr, ws_bytes, ctypes.byref(o), None) == 1
    o = _lib.default_options(schedule=5)
    assert lib.wg_upper_hood_ex(addr, 10, addr, addr, addr, ws_bytes, ctypes.byref(o), None) == 1
    # sort and unsorted input
    sws = lib.wg_sort_points_workspace_size(100)
    assert lib.wg_sort_points(addr, -1, addr, addr, addr, sws, None) == 1
    assert lib.wg_sort_points(addr, (1 << 30) + 1, addr, addr, addr, sws, None) == 7
    assert lib.wg_sort_points(addr, 10, None, addr, addr, sws, None) == 1
    assert lib.wg_sort_points(addr, 10, addr, None, addr, sws, None) == 1
    assert lib.wg_sort_points(addr + 4, 10, addr, addr, addr, sws, None) == 1
    assert lib.wg_sort_points(addr, 10, addr, addr, addr, 16, None) == 2
    assert lib.wg_sort_points(addr, 10, addr, addr, addr + 8, sws, None) == 1
    uws = lib.wg_upper_hood_unsorted_workspace_size(100)
    assert lib.wg_upper_hood_unsorted(addr, -1, addr, addr, addr, uws, None, None) == 1
    assert lib.wg_upper_hood_unsorted(addr, 10, addr, addr, addr, 16, None, None) == 2
    assert lib.wg_upper_hood_unsorted(addr, (1 << 30) + 1, addr, addr, addr, uws, None, None) == 7
    assert lib.wg_debug_bridge(addr, 0, addr, 1, addr, 0, None) == 1
    assert lib.wg_debug_warp_hood(addr, 33, addr, addr, 0, None) == 1
