"""CPU checks of the reasoning behind two steps of the GPU path, restated in
exact integer arithmetic and compared with the oracle's corner lists.

1. Neighbour pruning (the fused kernel's pending-list flush and the
   small-set kernel): an entry p of a list of distinct points in input order
   whose list neighbours a and b satisfy orient(a, p, b) >= 0 is not a
   corner; all of a round's deletions are made at once; a round that deletes
   nothing leaves a convex chain. Flushes see the survivors in chunks, the
   first entry of a chunk having the running hood's last corner as its left
   neighbour.
2. The single-column tile rule: on a tile whose points share one x, the
   column rule over the y's equals the general point rules.
They exercise the arguments, not the CUDA code, which the GPU parity tests
cover.
"""
import numpy as np
import pytest

import oracle
from paper_1203_5004_gb300 import inputs

KINDS = ["uniform", "arc", "band", "gauss_x", "gauss_disk", "columns", "duplicates"]


def orient(o, a, b):
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])


def survivors(kx, ky):
    """Height rule, then first occurrence and the column rule (the kernels'
    drop rules), over the whole set: the indices that remain, in order."""
    n = len(kx)
    P = list(zip(kx.tolist(), ky.tolist()))
    if n == 0:
        return P, []
    y = np.asarray(ky, dtype=np.int64)
    pre = np.full(n, -1, dtype=np.int64)
    suf = np.full(n, -1, dtype=np.int64)
    if n > 1:
        pre[1:] = np.maximum.accumulate(y[:-1])
        suf[:-1] = np.maximum.accumulate(y[::-1][:-1])[::-1]
    keep = []
    xfirst = P[0][0]
    for i in range(n):
        if pre[i] >= y[i] and suf[i] > y[i]:
            continue
        if i > 0 and P[i - 1] == P[i]:
            continue
        if i + 1 < n:
            nx, pv = P[i + 1], P[i - 1] if i > 0 else None
            if nx[0] == P[i][0] and nx[1] > P[i][1] and ((pv is not None and pv[0] == P[i][0]) or P[i][0] > xfirst):
                continue
        keep.append(i)
    return P, keep


def prune_rounds(P, L, anchor=None, max_rounds=10_000, strict_drop=False):
    """Rounds of neighbour pruning over list L until a round deletes nothing.
    anchor: the left neighbour of L[0] (a running hood's last corner)."""
    for _ in range(max_rounds):
        m = len(L)
        keep = []
        for e in range(m):
            a = P[L[e - 1]] if e > 0 else anchor
            drop = False
            if a is not None and e + 1 < m:
                o = orient(a, P[L[e]], P[L[e + 1]])
                drop = o > 0 if strict_drop else o >= 0
            if not drop:
                keep.append(L[e])
        if len(keep) == m:
            return L
        L = keep
    raise AssertionError("pruning did not converge")


def chain_merge(P, H, C):
    """Running hood H followed by the convex chain C: the hood of both (the
    monotone chain; the kernel finds the same chain with one bridge)."""
    out = list(H)
    for i in C:
        while len(out) >= 2 and orient(P[out[-2]], P[out[-1]], P[i]) >= 0:
            out.pop()
        out.append(i)
    return out


CASES = [(k, n, s) for k in KINDS for n, s in ((7, 1), (300, 2), (4096, 3), (20_000, 4))]


@pytest.mark.parametrize("kind,n,seed", CASES)
def test_pruning_rounds_reach_the_hood(kind, n, seed):
    ps = inputs.make(kind, n, seed)
    P, L = survivors(ps.kx, ps.ky)
    assert prune_rounds(P, L) == oracle.upper_hull(ps.kx, ps.ky).tolist()


@pytest.mark.parametrize("kind,n,seed", CASES)
def test_chunked_flushes_reach_the_hood(kind, n, seed):
    # the fused kernel's pending list: chunks of 128 survivors, each pruned
    # with the running hood's last corner as the first entry's neighbour,
    # then merged into the running hood
    ps = inputs.make(kind, n, seed)
    P, L = survivors(ps.kx, ps.ky)
    H = []
    for c0 in range(0, len(L), 128):
        chunk = prune_rounds(P, L[c0:c0 + 128], anchor=P[H[-1]] if H else None)
        H = chain_merge(P, H, chunk)
    assert H == oracle.upper_hull(ps.kx, ps.ky).tolist()


def test_planted_mistake_fails():
    # a plausible slip, dropping only strict left turns (so collinear points
    # stay), must disagree with the oracle somewhere
    wrong = 0
    for kind, n, seed in CASES:
        ps = inputs.make(kind, n, seed)
        P, L = survivors(ps.kx, ps.ky)
        wrong += prune_rounds(P, L, strict_drop=True) != oracle.upper_hull(ps.kx, ps.ky).tolist()
    assert wrong > 0


def point_rules(tile, prev, xfirst):
    """The general point rules on a tile (first occurrence, column rule);
    prev is the input point before the tile or None."""
    keep = []
    for j, p in enumerate(tile):
        pv = tile[j - 1] if j > 0 else prev
        d = pv is not None and pv == p
        if not d and j + 1 < len(tile):
            nx = tile[j + 1]
            d = nx[0] == p[0] and nx[1] > p[1] and ((pv is not None and pv[0] == p[0]) or p[0] > xfirst)
        keep.append(not d)
    return keep


def column_rules(tile, prev, xfirst):
    """The single-column tile rule over the y's (every x equal)."""
    x = tile[0][0]
    same_col = prev is not None and prev[0] == x
    yp = prev[1] if prev is not None else None
    keep = []
    for j, p in enumerate(tile):
        hn = j + 1 < len(tile)
        repeat = same_col and yp == p[1]
        up = hn and tile[j + 1][1] > p[1]
        keep.append(not (repeat or (up and (same_col or x > xfirst))))
        same_col, yp = True, p[1]
    return keep


def test_column_rules_equal_point_rules():
    r = np.random.default_rng(11)
    for trial in range(3000):
        x = int(r.integers(0, 8))
        m = int(r.integers(1, 40))
        ys = np.sort(r.integers(0, 12, size=m)).tolist()  # repeats included
        tile = [(x, y) for y in ys]
        xfirst = int(r.integers(0, x + 1))
        choice = int(r.integers(0, 4))
        if choice == 0:
            prev = None
        elif choice == 1:
            prev = (x, int(r.integers(0, ys[0] + 1)))  # same column, below or equal
        else:
            prev = (int(r.integers(0, x)) if x > 0 else None, int(r.integers(0, 12)))
            prev = None if prev[0] is None else prev
        assert column_rules(tile, prev, xfirst) == point_rules(tile, prev, xfirst), (tile, prev, xfirst)


@pytest.mark.parametrize("kind", KINDS)
def test_small_path_steps(kind):
    # the one-CTA small-set kernel: height rule over the whole set, the point
    # rules, pruning rounds; sizes up to its limit
    for n in (1, 2, 3, 16, 17, 511, 513, 4096, 8192):
        ps = inputs.make(kind, n, n + 5)
        P, L = survivors(ps.kx, ps.ky)
        assert prune_rounds(P, L) == oracle.upper_hull(ps.kx, ps.ky).tolist(), (kind, n)
