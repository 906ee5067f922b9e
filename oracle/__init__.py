"""CPU oracle for the upper hood (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and its reference arm) may import this package. The
product path never does: the CUDA library fails loudly instead of falling back
here.

``oracle.c`` holds the arithmetic (Andrew's monotone chain for the upper and
lower hoods, their O(n^3) brute forces, and the convex hull stitched from the
two chains, all with exact int64 orientation). ``strips.c`` runs the same chain on
contiguous strips in parallel threads and once more over the strip hoods (the
CPU baseline of the measurements). This module only compiles them with gcc,
loads them with ctypes and marshals numpy arrays.

``sort_points`` (the order of unsorted input) is one numpy call.

Parity status: every function here is pinned by ``tests/test_oracle.py``
(brute force, closed forms, Qhull in general position, invariants, Python
big-integer orientation; Python's own stable sort of coordinate pairs for
``sort_points``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "strips.c"))
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle sources into liboracle.so next to them (gcc, -O2, no -march)."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-pthread", "-shared", "-fPIC", "-o", tmp, *_SRCS])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i8p = ctypes.POINTER(ctypes.c_int8)
            lib.oracle_upper_hull.restype = ctypes.c_int64
            lib.oracle_upper_hull.argtypes = [i32p, i32p, ctypes.c_int64, i32p]
            lib.oracle_lower_hull.restype = ctypes.c_int64
            lib.oracle_lower_hull.argtypes = [i32p, i32p, ctypes.c_int64, i32p]
            lib.oracle_lower_hull_brute.restype = ctypes.c_int64
            lib.oracle_lower_hull_brute.argtypes = [i32p, i32p, ctypes.c_int64, i32p]
            lib.oracle_convex_hull.restype = ctypes.c_int64
            lib.oracle_convex_hull.argtypes = [i32p, i32p, ctypes.c_int64, i32p, i32p]
            lib.oracle_upper_hull_strips.restype = ctypes.c_int64
            lib.oracle_upper_hull_strips.argtypes = [i32p, i32p, ctypes.c_int64, i32p, ctypes.c_int]
            lib.oracle_upper_hull_batched_threads.restype = ctypes.c_int
            lib.oracle_upper_hull_batched_threads.argtypes = [i32p, i32p, i64p, ctypes.c_int64, i32p, i32p,
                                                              ctypes.c_int]
            lib.oracle_upper_hull_brute.restype = ctypes.c_int64
            lib.oracle_upper_hull_brute.argtypes = [i32p, i32p, ctypes.c_int64, i32p]
            lib.oracle_orient_sign.restype = ctypes.c_int
            lib.oracle_orient_sign.argtypes = [ctypes.c_int32] * 6
            lib.oracle_orient_signs.restype = None
            lib.oracle_orient_signs.argtypes = [i32p, i32p, ctypes.c_int64, i8p]
            lib.oracle_upper_hull_batched.restype = None
            lib.oracle_upper_hull_batched.argtypes = [i32p, i32p, i64p, ctypes.c_int64, i32p, i32p]
            _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _ints(kx, ky):
    kx = np.ascontiguousarray(kx, dtype=np.int32)
    ky = np.ascontiguousarray(ky, dtype=np.int32)
    if kx.shape != ky.shape or kx.ndim != 1:
        raise ValueError("kx and ky must be 1-D arrays of equal length")
    return kx, ky


def upper_hull(kx, ky) -> np.ndarray:
    """Indices of the strict upper-hood corners, left to right (monotone chain)."""
    kx, ky = _ints(kx, ky)
    out = np.empty(max(1, kx.shape[0]), dtype=np.int32)
    h = _load().oracle_upper_hull(_p(kx, ctypes.c_int32), _p(ky, ctypes.c_int32),
                                  kx.shape[0], _p(out, ctypes.c_int32))
    return out[:h].copy()


def lower_hull(kx, ky) -> np.ndarray:
    """Indices of the strict lower-hood corners, left to right (monotone chain)."""
    kx, ky = _ints(kx, ky)
    out = np.empty(max(1, kx.shape[0]), dtype=np.int32)
    h = _load().oracle_lower_hull(_p(kx, ctypes.c_int32), _p(ky, ctypes.c_int32),
                                  kx.shape[0], _p(out, ctypes.c_int32))
    return out[:h].copy()


def lower_hull_brute(kx, ky) -> np.ndarray:
    """Same set by the O(n^3) witness-pair definition (small n only)."""
    kx, ky = _ints(kx, ky)
    if kx.shape[0] > 2048:
        raise ValueError("brute force is O(n^3); keep n small")
    out = np.empty(max(1, kx.shape[0]), dtype=np.int32)
    h = _load().oracle_lower_hull_brute(_p(kx, ctypes.c_int32), _p(ky, ctypes.c_int32),
                                        kx.shape[0], _p(out, ctypes.c_int32))
    return out[:h].copy()


def convex_hull(kx, ky) -> np.ndarray:
    """Convex-hull corners clockwise from the first point: upper hood, then the
    lower hood back without its ends."""
    kx, ky = _ints(kx, ky)
    n = kx.shape[0]
    out = np.empty(max(1, n), dtype=np.int32)
    scratch = np.empty(max(1, n), dtype=np.int32)
    h = _load().oracle_convex_hull(_p(kx, ctypes.c_int32), _p(ky, ctypes.c_int32), n,
                                   _p(out, ctypes.c_int32), _p(scratch, ctypes.c_int32))
    return out[:h].copy()


def upper_hull_strips(kx, ky, threads: int | None = None) -> np.ndarray:
    """The same corners by the strip-parallel chain on `threads` host threads (default: all cores)."""
    kx, ky = _ints(kx, ky)
    t = int(threads) if threads else (os.cpu_count() or 1)
    out = np.empty(max(1, kx.shape[0]), dtype=np.int32)
    h = _load().oracle_upper_hull_strips(_p(kx, ctypes.c_int32), _p(ky, ctypes.c_int32),
                                         kx.shape[0], _p(out, ctypes.c_int32), t)
    if h < 0:
        raise MemoryError("oracle_upper_hull_strips: out of memory or threads")
    return out[:h].copy()


def sort_points(kx, ky) -> np.ndarray:
    """The order of points given in any order, sorted by (x, y) and stable
    (the step before the path: Section 2 takes its points sorted): perm with
    (kx, ky)[perm] sorted lexicographically and equal points in input order.
    One library step, numpy's stable sort of the 48-bit keys kx 2^24 + ky
    (which order grid points exactly as (x, y))."""
    kx = np.asarray(kx, dtype=np.int64)
    ky = np.asarray(ky, dtype=np.int64)
    return np.argsort((kx << 24) | ky, kind="stable").astype(np.int32)


def upper_hull_brute(kx, ky) -> np.ndarray:
    """Same set by the O(n^3) witness-pair definition (small n only)."""
    kx, ky = _ints(kx, ky)
    if kx.shape[0] > 2048:
        raise ValueError("brute force is O(n^3); keep n small")
    out = np.empty(max(1, kx.shape[0]), dtype=np.int32)
    h = _load().oracle_upper_hull_brute(_p(kx, ctypes.c_int32), _p(ky, ctypes.c_int32),
                                        kx.shape[0], _p(out, ctypes.c_int32))
    return out[:h].copy()


def orient_sign(o, a, b) -> int:
    """sign(det(a - o, b - o)) for integer grid points given as (kx, ky) pairs."""
    return int(_load().oracle_orient_sign(int(o[0]), int(o[1]), int(a[0]), int(a[1]),
                                          int(b[0]), int(b[1])))


def orient_signs(kx, ky) -> np.ndarray:
    """Signs for consecutive triples (3t, 3t+1, 3t+2) of the given points."""
    kx, ky = _ints(kx, ky)
    if kx.shape[0] % 3:
        raise ValueError("need a multiple of 3 points")
    out = np.empty(kx.shape[0] // 3, dtype=np.int8)
    _load().oracle_orient_signs(_p(kx, ctypes.c_int32), _p(ky, ctypes.c_int32),
                                out.shape[0], _p(out, ctypes.c_int8))
    return out


def upper_hull_batched(kx, ky, offsets):
    """Per-set corners: returns (out, counts) with set s at out[offsets[s]:offsets[s]+counts[s]]."""
    kx, ky = _ints(kx, ky)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    num_sets = offsets.shape[0] - 1
    out = np.empty(max(1, kx.shape[0]), dtype=np.int32)
    counts = np.empty(max(1, num_sets), dtype=np.int32)
    _load().oracle_upper_hull_batched(_p(kx, ctypes.c_int32), _p(ky, ctypes.c_int32),
                                      _p(offsets, ctypes.c_int64), num_sets,
                                      _p(out, ctypes.c_int32), _p(counts, ctypes.c_int32))
    return out, counts[:num_sets].copy()


def upper_hull_batched_threads(kx, ky, offsets, threads: int | None = None):
    """The batched form with the sets spread over `threads` host threads (default: all cores)."""
    kx, ky = _ints(kx, ky)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    num_sets = offsets.shape[0] - 1
    t = int(threads) if threads else (os.cpu_count() or 1)
    out = np.empty(max(1, kx.shape[0]), dtype=np.int32)
    counts = np.empty(max(1, num_sets), dtype=np.int32)
    if _load().oracle_upper_hull_batched_threads(_p(kx, ctypes.c_int32), _p(ky, ctypes.c_int32),
                                                 _p(offsets, ctypes.c_int64), num_sets,
                                                 _p(out, ctypes.c_int32), _p(counts, ctypes.c_int32), t) != 0:
        raise RuntimeError("oracle_upper_hull_batched_threads: could not start threads")
    return out, counts[:num_sets].copy()


def bridge(p_kx, p_ky, q_kx, q_ky):
    """Bridge (upper common tangent) of two hoods P and Q, P entirely lex-left of Q.

    Defined from the merged hood (paper Section 2, match_and_merge outline):
    H(P u Q) = P[0..p] ++ Q[q..], so p is the last corner of the merged hood
    that comes from P and q the first that comes from Q. Returns (p, q), with
    -1 for a side that contributes nothing.
    """
    kx = np.concatenate([np.asarray(p_kx, np.int32), np.asarray(q_kx, np.int32)])
    ky = np.concatenate([np.asarray(p_ky, np.int32), np.asarray(q_ky, np.int32)])
    hp = len(p_kx)
    h = upper_hull(kx, ky)
    from_p = h[h < hp]
    from_q = h[h >= hp]
    p = int(from_p[-1]) if from_p.size else -1
    q = int(from_q[0]) - hp if from_q.size else -1
    return p, q
