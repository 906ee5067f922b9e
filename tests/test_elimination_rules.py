"""CPU checks of the exactness arguments behind the GPU path's pre-filters.

The fused kernel drops points before any hood work by three rules and
decides many orientations in float32 without a float64 pass. Each rule is
claimed to drop only points that cannot be corners; these tests restate
each rule on the CPU (float32 arithmetic through numpy, one rounding per
operation, no fused multiply-add) and check it against the oracle's corner
lists: no corner may ever be dropped. They exercise the reasoning, not the
CUDA code, which the GPU parity tests cover.
"""
import numpy as np
import pytest

import oracle
from paper_1203_5004_gb300 import inputs

F32 = np.float32


def _pts(kind, n, seed):
    ps = inputs.make(kind, n, seed)
    return ps, ps.points().astype(F32)


CASES = [("uniform", 1 << 14, 1), ("band", 1 << 15, 2), ("arc", 1 << 14, 3), ("gauss_x", 1 << 15, 4),
         ("columns", 5000, 5), ("duplicates", 4000, 6), ("gauss_disk", 1 << 14, 7)]


def _dropped_by_heights(lo, hi):
    """Indices i with max(lo[:i]) >= hi[i] and max(lo[i+1:]) > hi[i]."""
    n = lo.shape[0]
    pre = np.full(n, -np.inf, dtype=F32)
    suf = np.full(n, -np.inf, dtype=F32)
    if n > 1:
        pre[1:] = np.maximum.accumulate(lo[:-1])
        suf[:-1] = np.maximum.accumulate(lo[::-1][:-1])[::-1]
    return np.nonzero((pre >= hi) & (suf > hi))[0]


@pytest.mark.parametrize("kind,n,seed", CASES)
def test_height_rule_drops_no_corner(kind, n, seed):
    ps, p = _pts(kind, n, seed)
    corners = set(oracle.upper_hull(ps.kx, ps.ky).tolist())
    y = p[:, 1]
    dropped = _dropped_by_heights(y, y)
    assert not corners.intersection(dropped.tolist())


def _sheared_bounds(p, x0, y0, s):
    """The kernel's sheared heights as float32 intervals (one rounding per
    operation): t = s (x - x0), y' = (y - y0) - t, e = 2^-22 (|t| + |y'|)."""
    x, y = p[:, 0], p[:, 1]
    t = (F32(s) * (x - F32(x0))).astype(F32)
    yp = ((y - F32(y0)).astype(F32) - t).astype(F32)
    ec = F32(2.0 ** -22) if s != 0 else F32(0)
    e = ((np.abs(t) + np.abs(yp)).astype(F32) * ec).astype(F32)
    return (yp - e).astype(F32), (yp + e).astype(F32)


@pytest.mark.parametrize("kind,n,seed", CASES)
def test_sheared_rule_drops_no_corner(kind, n, seed):
    ps, p = _pts(kind, n, seed)
    corners = set(oracle.upper_hull(ps.kx, ps.ky).tolist())
    r = np.random.default_rng(seed)
    for trial in range(40):
        # a window of consecutive points, sheared by its chord slope (as the
        # kernel does per tile) or by an integer / random slope
        a = int(r.integers(0, n - 2))
        b = int(min(n, a + r.integers(2, 2000)))
        w = p[a:b]
        f0, f1 = w[0], w[-1]
        mode = trial % 3
        if mode == 0:
            s = F32((f1[1] - f0[1]) / (f1[0] - f0[0])) if f1[0] > f0[0] else F32(0)
        elif mode == 1:
            s = F32(int(r.integers(-8, 9)))
        else:
            s = F32(r.normal(0, 100))
        if not np.abs(s) < 1e6:
            s = F32(0)
        lo, hi = _sheared_bounds(w, f0[0], f0[1], s)
        dropped = _dropped_by_heights(lo, hi) + a
        assert not corners.intersection(dropped.tolist()), (kind, trial, float(s))


@pytest.mark.parametrize("kind,n,seed", CASES)
def test_column_rule_drops_no_corner(kind, n, seed):
    ps, p = _pts(kind, n, seed)
    corners = set(oracle.upper_hull(ps.kx, ps.ky).tolist())
    x, y = p[:, 0], p[:, 1]
    i = np.arange(0, n - 1)
    up = (x[i + 1] == x[i]) & (y[i + 1] > y[i])
    below = np.zeros(i.shape, dtype=bool)  # a point before i in its column
    below[1:] = x[i[1:] - 1] == x[i[1:]]
    left = below | (x[i] > x[0])
    dropped = i[up & left]
    assert not corners.intersection(dropped.tolist())


def test_small_products_are_exact_in_float32():
    # orient(o, a, b) with all differences below 2^11 grid units: when both
    # float32 products are below 2^-25, the float32 determinant equals the
    # exact one (zero included)
    r = np.random.default_rng(9)
    n = 200_000
    o = r.integers(0, inputs.G - (1 << 12), size=(n, 2))
    a = o + r.integers(-(1 << 11), 1 << 11, size=(n, 2))
    b = o + r.integers(-(1 << 11), 1 << 11, size=(n, 2))
    a, b = np.clip(a, 0, inputs.G - 1), np.clip(b, 0, inputs.G - 1)
    exact = (a[:, 0] - o[:, 0]) * (b[:, 1] - o[:, 1]) - (a[:, 1] - o[:, 1]) * (b[:, 0] - o[:, 0])
    u = F32(2.0 ** -24)
    fo, fa, fb = o.astype(F32) * u, a.astype(F32) * u, b.astype(F32) * u
    dx1, dy1 = (fa[:, 0] - fo[:, 0]).astype(F32), (fa[:, 1] - fo[:, 1]).astype(F32)
    dx2, dy2 = (fb[:, 0] - fo[:, 0]).astype(F32), (fb[:, 1] - fo[:, 1]).astype(F32)
    t1, t2 = (dx1 * dy2).astype(F32), (dy1 * dx2).astype(F32)
    d = (t1 - t2).astype(F32)
    small = np.maximum(np.abs(t1), np.abs(t2)) < F32(2.0 ** -25)
    assert small.mean() > 0.9
    assert np.array_equal(np.sign(d[small]).astype(np.int64), np.sign(exact[small]))
    # and the float32 determinant is the exact value, scaled
    assert np.array_equal(d[small].astype(np.float64) * 2.0 ** 48, exact[small].astype(np.float64))


def test_sheared_rule_keeps_bumps_on_steep_lines():
    # Steep exact lines with a one-unit bump, sheared by the float32 value of
    # their slope: the bump is a corner, strictly above the chord of the
    # others, while the heights of the points on the line are equal in exact
    # arithmetic and differ only by rounding. The bump must be kept.
    r = np.random.default_rng(10)
    u = 2.0 ** -24
    for trial in range(200):
        q = int(r.integers(1, 16))
        pnum = int(r.integers(500 * q, 2000 * q))
        m = int(r.integers(20, 200))
        k = np.arange(m, dtype=np.int64)
        kx = 1000 + k * q
        ky = 1000 + k * pnum
        assert ky[-1] < inputs.G
        j = int(r.integers(1, m - 1))
        ky = ky.copy()
        ky[j] += 1
        corners = set(oracle.upper_hull(kx, ky).tolist())
        assert j in corners
        p = inputs.to_float_points(kx, ky).astype(F32)
        s = F32(pnum / q)
        lo, hi = _sheared_bounds(p, p[0, 0], p[0, 1], s)
        dropped = _dropped_by_heights(lo, hi)
        assert not corners.intersection(dropped.tolist()), (trial, q, pnum, j)
