"""Python face of libwagener: the same entry points as include/wg.h.

Tensors carry device memory and the current CUDA stream; every step of the
computation runs in the library's kernels. Functions raise WagenerError on a
non-OK status.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import Options, WagenerError, check, default_options, load  # noqa: F401


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else int(t.data_ptr())


def _as_points(points: torch.Tensor) -> torch.Tensor:
    if points.dtype != torch.float32 or not points.is_cuda:
        raise TypeError("points must be a float32 CUDA tensor of shape (n, 2)")
    if points.dim() != 2 or points.shape[1] != 2 or not points.is_contiguous():
        raise ValueError("points must be a contiguous (n, 2) tensor")
    return points


def workspace_size(n: int) -> int:
    return int(load().wg_upper_hood_workspace_size(int(n)))


def plain_workspace_size(n: int) -> int:
    return int(load().wg_upper_hood_plain_workspace_size(int(n)))


def batched_workspace_size(offsets_host: np.ndarray) -> int:
    off = np.ascontiguousarray(offsets_host, dtype=np.int64)
    return int(load().wg_upper_hood_batched_workspace_size(off.ctypes.data, off.shape[0] - 1))


def new_workspace(nbytes: int, device=None) -> torch.Tensor:
    """A zero-filled workspace (zeroed once; the library keeps it reusable)."""
    return torch.zeros(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def upper_hood_into(points: torch.Tensor, out_idx: torch.Tensor, out_count: torch.Tensor,
                    workspace: torch.Tensor, opts: Options | None = None, stream=None) -> None:
    """wg_upper_hood_ex on caller-owned buffers (no allocation, no sync)."""
    points = _as_points(points)
    n = points.shape[0]
    code = load().wg_upper_hood_ex(_ptr(points), n, _ptr(out_idx), _ptr(out_count), _ptr(workspace),
                                   workspace.numel(), ctypes.byref(opts) if opts else None, _stream(stream))
    check(code, "wg_upper_hood_ex")


def upper_hood(points: torch.Tensor, opts: Options | None = None, workspace: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """Indices (int32, on the device) of the upper-hood corners of sorted grid points."""
    points = _as_points(points)
    n = points.shape[0]
    dev = points.device
    ws = workspace if workspace is not None else new_workspace(workspace_size(n), dev)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    upper_hood_into(points, out, cnt, ws, opts, stream)
    return out[: int(cnt.item())]


def convex_hull_workspace_size(n: int) -> int:
    return int(load().wg_convex_hull_workspace_size(int(n)))


def convex_hull_into(points: torch.Tensor, out_idx: torch.Tensor, out_count: torch.Tensor,
                     workspace: torch.Tensor, opts: Options | None = None, stream=None) -> None:
    """wg_convex_hull on caller-owned buffers (no allocation, no sync)."""
    points = _as_points(points)
    n = points.shape[0]
    code = load().wg_convex_hull(_ptr(points), n, _ptr(out_idx), _ptr(out_count), _ptr(workspace),
                                 workspace.numel(), ctypes.byref(opts) if opts else None, _stream(stream))
    check(code, "wg_convex_hull")


def convex_hull(points: torch.Tensor, opts: Options | None = None, workspace: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """Indices (int32, on the device) of the convex-hull corners, clockwise from the first point."""
    points = _as_points(points)
    n = points.shape[0]
    dev = points.device
    ws = workspace if workspace is not None else new_workspace(convex_hull_workspace_size(n), dev)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    convex_hull_into(points, out, cnt, ws, opts, stream)
    return out[: int(cnt.item())]


def sort_points_workspace_size(n: int) -> int:
    return int(load().wg_sort_points_workspace_size(int(n)))


def sort_points(points: torch.Tensor, workspace: torch.Tensor | None = None, stream=None):
    """Grid points in any order sorted by (x, y) on the device, stably: returns
    (sorted points float32 (n, 2), perm int32 (n,)) with sorted[i] = points[perm[i]]."""
    points = _as_points(points)
    n = points.shape[0]
    dev = points.device
    ws = workspace if workspace is not None else new_workspace(sort_points_workspace_size(n), dev)
    out = torch.empty((max(n, 1), 2), dtype=torch.float32, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    check(load().wg_sort_points(_ptr(points), n, _ptr(out), _ptr(perm), _ptr(ws), ws.numel(), _stream(stream)),
          "wg_sort_points")
    return out[:n], perm[:n]


def upper_hood_unsorted_workspace_size(n: int) -> int:
    return int(load().wg_upper_hood_unsorted_workspace_size(int(n)))


def upper_hood_unsorted(points: torch.Tensor, opts: Options | None = None, workspace: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
    """Indices (int32, on the device, into the input order) of the upper-hood
    corners of grid points given in any order."""
    points = _as_points(points)
    n = points.shape[0]
    dev = points.device
    ws = workspace if workspace is not None else new_workspace(upper_hood_unsorted_workspace_size(n), dev)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    check(load().wg_upper_hood_unsorted(_ptr(points), n, _ptr(out), _ptr(cnt), _ptr(ws), ws.numel(),
                                        ctypes.byref(opts) if opts else None, _stream(stream)),
          "wg_upper_hood_unsorted")
    return out[: int(cnt.item())]


def upper_hood_plain(points: torch.Tensor, opts: Options | None = None, workspace: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    """Same result by the unfused schedule (one launch per stage)."""
    points = _as_points(points)
    n = points.shape[0]
    dev = points.device
    ws = workspace if workspace is not None else new_workspace(plain_workspace_size(n), dev)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    code = load().wg_upper_hood_plain(_ptr(points), n, _ptr(out), _ptr(cnt), _ptr(ws), ws.numel(),
                                      ctypes.byref(opts) if opts else None, _stream(stream))
    check(code, "wg_upper_hood_plain")
    return out[: int(cnt.item())]


def upper_hood_batched_into(points: torch.Tensor, offsets: torch.Tensor, out_idx: torch.Tensor,
                            out_counts: torch.Tensor, workspace: torch.Tensor, opts: Options | None = None,
                            stream=None) -> None:
    num_sets = offsets.shape[0] - 1
    code = load().wg_upper_hood_batched(_ptr(points), _ptr(offsets), num_sets, _ptr(out_idx), _ptr(out_counts),
                                        _ptr(workspace), workspace.numel(),
                                        ctypes.byref(opts) if opts else None, _stream(stream))
    check(code, "wg_upper_hood_batched")


def upper_hood_batched(points: torch.Tensor, offsets_host: np.ndarray, opts: Options | None = None,
                       stream=None):
    """Per-set hoods: returns (out_idx, out_counts) on the device, CSR-aligned."""
    points = _as_points(points)
    dev = points.device
    off_h = np.ascontiguousarray(offsets_host, dtype=np.int64)
    offsets = torch.from_numpy(off_h).to(dev)
    ws = new_workspace(batched_workspace_size(off_h), dev)
    out = torch.empty(max(int(off_h[-1]), 1), dtype=torch.int32, device=dev)
    counts = torch.empty(max(off_h.shape[0] - 1, 1), dtype=torch.int32, device=dev)
    upper_hood_batched_into(points, offsets, out, counts, ws, opts, stream)
    return out, counts[: off_h.shape[0] - 1]


def upper_hood_from_host(points_host: np.ndarray, d_points: torch.Tensor, d_out: torch.Tensor,
                         d_count: torch.Tensor, workspace: torch.Tensor, h_out: np.ndarray,
                         opts: Options | None = None, stream=None) -> int:
    """Host (n, 2) float32 in, host corner indices out (h_out[:count]); returns count."""
    n = points_host.shape[0]
    h_cnt = np.zeros(1, dtype=np.int32)
    code = load().wg_upper_hood_from_host(points_host.ctypes.data, n, h_out.ctypes.data, h_cnt.ctypes.data,
                                          _ptr(d_points), _ptr(d_out), _ptr(d_count), _ptr(workspace),
                                          workspace.numel(), ctypes.byref(opts) if opts else None,
                                          _stream(stream))
    check(code, "wg_upper_hood_from_host")
    return int(h_cnt[0])


def device_status(workspace: torch.Tensor, stream=None) -> int:
    return int(load().wg_get_device_status(_ptr(workspace), _stream(stream)))


def read_counters(workspace: torch.Tensor, stream=None) -> tuple[int, int]:
    t = ctypes.c_uint64()
    f = ctypes.c_uint64()
    check(load().wg_read_counters(_ptr(workspace), ctypes.byref(t), ctypes.byref(f), _stream(stream)),
          "wg_read_counters")
    return int(t.value), int(f.value)


def autotune(points: torch.Tensor, workspace: torch.Tensor | None = None, stream=None) -> Options:
    points = _as_points(points)
    n = points.shape[0]
    dev = points.device
    ws = workspace if workspace is not None else new_workspace(workspace_size(n), dev)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    best = Options()
    check(load().wg_autotune(_ptr(points), n, _ptr(out), _ptr(cnt), _ptr(ws), ws.numel(), ctypes.byref(best),
                             _stream(stream)), "wg_autotune")
    return best


def autotune_batched(points: torch.Tensor, offsets: torch.Tensor, workspace: torch.Tensor, stream=None) -> Options:
    """wg_autotune_batched on the caller's sets (offsets: device int64 CSR)."""
    points = _as_points(points)
    num_sets = offsets.shape[0] - 1
    total = points.shape[0]
    out = torch.empty(max(total, 1), dtype=torch.int32, device=points.device)
    counts = torch.empty(max(num_sets, 1), dtype=torch.int32, device=points.device)
    best = Options()
    check(load().wg_autotune_batched(_ptr(points), _ptr(offsets), num_sets, _ptr(out), _ptr(counts),
                                     _ptr(workspace), workspace.numel(), ctypes.byref(best), _stream(stream)),
          "wg_autotune_batched")
    return best


def debug_orient(triples: torch.Tensor, pred_mode: int = _lib.WG_PRED_FILTERED, stream=None):
    """Signs of orient for consecutive point triples; returns (signs int8, fallbacks)."""
    triples = _as_points(triples)
    ntri = triples.shape[0] // 3
    signs = torch.empty(max(ntri, 1), dtype=torch.int8, device=triples.device)
    fb = torch.zeros(1, dtype=torch.int64, device=triples.device)
    check(load().wg_debug_orient(_ptr(triples), ntri, _ptr(signs), _ptr(fb), pred_mode, _stream(stream)),
          "wg_debug_orient")
    return signs[:ntri], int(fb.item())


def debug_bridge(P: torch.Tensor, Q: torch.Tensor, pred_mode: int = _lib.WG_PRED_FILTERED, stream=None):
    out = torch.empty(2, dtype=torch.int32, device=P.device)
    check(load().wg_debug_bridge(_ptr(_as_points(P)), P.shape[0], _ptr(_as_points(Q)), Q.shape[0], _ptr(out),
                                 pred_mode, _stream(stream)), "wg_debug_bridge")
    r = out.cpu().tolist()
    return r[0], r[1]


def debug_bridge_cta(P: torch.Tensor, Q: torch.Tensor, pred_mode: int = _lib.WG_PRED_FILTERED, stream=None):
    out = torch.empty(2, dtype=torch.int32, device=P.device)
    check(load().wg_debug_bridge_cta(_ptr(_as_points(P)), P.shape[0], _ptr(_as_points(Q)), Q.shape[0], _ptr(out),
                                     pred_mode, _stream(stream)), "wg_debug_bridge_cta")
    r = out.cpu().tolist()
    return r[0], r[1]


def debug_warp_hood(points: torch.Tensor, pred_mode: int = _lib.WG_PRED_FILTERED, stream=None):
    m = points.shape[0]
    out = torch.empty(32, dtype=torch.int32, device=points.device)
    cnt = torch.empty(1, dtype=torch.int32, device=points.device)
    check(load().wg_debug_warp_hood(_ptr(_as_points(points)) if m else None, m, _ptr(out), _ptr(cnt), pred_mode,
                                    _stream(stream)), "wg_debug_warp_hood")
    return out[: int(cnt.item())].cpu().numpy()


def debug_set_stall(workspace: torch.Tensor, stall_ns: int, stream=None) -> None:
    check(load().wg_debug_set_stall(_ptr(workspace), int(stall_ns), _stream(stream)), "wg_debug_set_stall")
