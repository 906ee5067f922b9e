"""Seeded synthetic point sets for the upper-hood path (shared input generators).

This module only draws and sorts random grid points; it contains none of the
hull arithmetic. Both the CUDA path and the CPU oracle receive its output, so
the two sides always see identical inputs.

Coordinate model. A point is (x, y) = (kx * 2^-24, ky * 2^-24) with integers
kx, ky in [0, 2^24). Such values are exact in float32 (24-bit integers times a
power of two) and every difference of two of them is exact too. Sets are sorted
lexicographically by (x, y), i.e. by the integer key kx * 2^24 + ky, which is
the left-to-right order the paper assumes for its input (Section 2).

The workloads are synthetic stand-ins shaped like the paper's setting (no
public dataset is involved):

* ``uniform``      kx, ky uniform in [0, 2^24)
* ``arc``          kx uniform, y = 1 - 4 (x - 1/2)^2 rounded down to the grid
                   (the apex y = 1 is clamped to the last grid row)
* ``band``         the arc plus a uniform integer offset in [-8, 8) grid units
                   (a band 2^-20 wide), clamped to the grid
* ``closed_form``  x = i 2^-12, y = i (4095 - i) 2^-24 for i < 4096: a strictly
                   concave integer sequence, so every point is a corner
* ``gauss_x``      x ~ N(1/2, 0.15) clipped to [0, 1), y uniform (many repeated
                   x values, so vertical runs and duplicate points occur)
* ``gauss_disk``   both coordinates ~ N(1/2, 0.15), clipped to [0, 1)
"""
from __future__ import annotations

import math

import numpy as np

GRID_BITS = 24
G = 1 << GRID_BITS            # grid cells per unit
U = 2.0 ** -GRID_BITS          # grid spacing = float32 unit roundoff

__all__ = [
    "G", "U", "PointSet", "to_float_points", "sort_lex",
    "uniform", "arc", "band", "closed_form", "gauss_x", "gauss_disk",
    "columns", "duplicates", "make", "batched_sizes", "batched",
]


class PointSet:
    """Sorted integer grid coordinates plus the float32 (n, 2) array the GPU reads."""

    __slots__ = ("kx", "ky", "name")

    def __init__(self, kx: np.ndarray, ky: np.ndarray, name: str = ""):
        self.kx = np.ascontiguousarray(kx, dtype=np.int32)
        self.ky = np.ascontiguousarray(ky, dtype=np.int32)
        self.name = name

    def __len__(self) -> int:
        return int(self.kx.shape[0])

    def points(self) -> np.ndarray:
        return to_float_points(self.kx, self.ky)


def to_float_points(kx: np.ndarray, ky: np.ndarray) -> np.ndarray:
    """(n, 2) float32 array of (kx * 2^-24, ky * 2^-24); exact for 24-bit integers."""
    out = np.empty((kx.shape[0], 2), dtype=np.float32)
    scale = np.float32(U)
    np.multiply(kx.astype(np.float32), scale, out=out[:, 0])
    np.multiply(ky.astype(np.float32), scale, out=out[:, 1])
    return out


def sort_lex(kx: np.ndarray, ky: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Sort by (kx, ky) through the 48-bit key kx * 2^24 + ky."""
    key = (kx.astype(np.int64) << GRID_BITS) | ky.astype(np.int64)
    key.sort()
    return (key >> GRID_BITS).astype(np.int32), (key & (G - 1)).astype(np.int32)


def _rng(seed) -> np.random.Generator:
    if isinstance(seed, np.random.Generator):
        return seed
    return np.random.Generator(np.random.PCG64(seed))


def _clip_grid(v: np.ndarray) -> np.ndarray:
    return np.clip(v, 0, G - 1).astype(np.int32)


def _arc_ky(kx: np.ndarray) -> np.ndarray:
    # floor(G * (1 - 4 (x - 1/2)^2)) = G - ceil((kx - 2^23)^2 / 2^22), clamped.
    d = kx.astype(np.int64) - (1 << 23)
    sq = d * d
    ceil_div = (sq + (1 << 22) - 1) >> 22
    return np.minimum(G - 1, G - ceil_div).astype(np.int64)


def uniform(n: int, seed=7) -> PointSet:
    r = _rng(seed)
    kx = r.integers(0, G, size=n, dtype=np.int64)
    ky = r.integers(0, G, size=n, dtype=np.int64)
    return PointSet(*sort_lex(kx, ky), name=f"uniform_n{n}")


def arc(n: int, seed=3) -> PointSet:
    r = _rng(seed)
    kx = np.sort(r.integers(0, G, size=n, dtype=np.int64))
    ky = _arc_ky(kx)
    return PointSet(*sort_lex(kx, ky), name=f"arc_n{n}")


def band(n: int, seed=4) -> PointSet:
    r = _rng(seed)
    kx = r.integers(0, G, size=n, dtype=np.int64)
    off = r.integers(-8, 8, size=n, dtype=np.int64)
    ky = _clip_grid(_arc_ky(kx) + off)
    return PointSet(*sort_lex(kx, ky), name=f"band_n{n}")


def closed_form() -> PointSet:
    i = np.arange(4096, dtype=np.int64)
    kx = i << 12
    ky = i * (4095 - i)
    return PointSet(kx, ky, name="closed_form_n4096")


def _gauss_grid(r: np.random.Generator, n: int) -> np.ndarray:
    v = r.normal(0.5, 0.15, size=n)
    v = np.clip(v, 0.0, 1.0 - U)
    return np.floor(v * G).astype(np.int64)


def gauss_x(n: int, seed=6) -> PointSet:
    r = _rng(seed)
    kx = _gauss_grid(r, n)
    ky = r.integers(0, G, size=n, dtype=np.int64)
    return PointSet(*sort_lex(kx, ky), name=f"gauss_x_n{n}")


def gauss_disk(n: int, seed=5) -> PointSet:
    r = _rng(seed)
    kx = _gauss_grid(r, n)
    ky = _gauss_grid(r, n)
    return PointSet(*sort_lex(kx, ky), name=f"gauss_disk_n{n}")


def columns(n: int, seed=11, ncols: int = 4, span: int = 64) -> PointSet:
    """Few distinct x values, small y range: many vertical runs and repeats."""
    r = _rng(seed)
    xs = r.integers(0, G, size=max(1, ncols), dtype=np.int64)
    kx = xs[r.integers(0, xs.shape[0], size=n)]
    ky = r.integers(0, span, size=n, dtype=np.int64) * (G // span)
    return PointSet(*sort_lex(kx, ky), name=f"columns_n{n}")


def duplicates(n: int, seed=12, distinct: int = 16, span: int = 256) -> PointSet:
    """Points drawn from a small pool on a coarse lattice: exact repeats everywhere."""
    r = _rng(seed)
    pool_x = r.integers(0, span, size=distinct, dtype=np.int64) * (G // span)
    pool_y = r.integers(0, span, size=distinct, dtype=np.int64) * (G // span)
    pick = r.integers(0, distinct, size=n)
    return PointSet(*sort_lex(pool_x[pick], pool_y[pick]), name=f"dups_n{n}")


_GENERATORS = {
    "uniform": uniform, "arc": arc, "band": band, "gauss_x": gauss_x,
    "gauss_disk": gauss_disk, "columns": columns, "duplicates": duplicates,
}


def make(kind: str, n: int, seed) -> PointSet:
    if kind == "closed_form":
        return closed_form()
    return _GENERATORS[kind](n, seed)


# ---------------------------------------------------------------------------
# Batched workload: many independent sets with log-uniform sizes.
# ---------------------------------------------------------------------------

BATCH_KINDS = ("uniform", "gauss_disk", "band")


def batched_sizes(num_sets: int, seed=5, lo: int = 3, hi: int = 65536) -> np.ndarray:
    """Sizes floor(exp(U(ln lo, ln(hi + 1)))) clamped to [lo, hi] (not powers of two)."""
    r = _rng(np.random.SeedSequence(seed).spawn(1)[0])
    s = np.floor(np.exp(r.uniform(math.log(lo), math.log(hi + 1), size=num_sets)))
    return np.clip(s, lo, hi).astype(np.int64)


def batched(num_sets: int, seed=5, lo: int = 3, hi: int = 65536):
    """Return (PointSet of all points concatenated, int64 CSR offsets, kinds).

    Set s draws its kind uniformly from BATCH_KINDS and its points from its own
    child seed, so any set can be regenerated independently of the others.
    """
    sizes = batched_sizes(num_sets, seed, lo, hi)
    offsets = np.zeros(num_sets + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    kx = np.empty(total, dtype=np.int32)
    ky = np.empty(total, dtype=np.int32)
    kinds = np.empty(num_sets, dtype=np.int8)
    children = np.random.SeedSequence(seed).spawn(num_sets + 1)[1:]
    for s in range(num_sets):
        r = _rng(children[s])
        kind = int(r.integers(0, len(BATCH_KINDS)))
        kinds[s] = kind
        ps = _GENERATORS[BATCH_KINDS[kind]](int(sizes[s]), r)
        a, b = offsets[s], offsets[s + 1]
        kx[a:b] = ps.kx
        ky[a:b] = ps.ky
    return PointSet(kx, ky, name=f"batched_S{num_sets}"), offsets, kinds
