"""Pins for the CPU oracle (no GPU needed).

The oracle (Andrew's monotone chain, exact int64 orientation) is checked
against things other than itself:
  * an independent O(n^3) definition (witness pairs) on small inputs of every
    generator, including repeats, columns and collinear runs;
  * closed forms (strictly concave and strictly convex integer parabolas,
    collinear lines, single columns, repeats);
  * Qhull (scipy.spatial.ConvexHull) on inputs in general position;
  * hand-derived cases under tests/golden/;
  * invariants on large inputs, checked by code written for the test;
  * Python big-integer orientation signs;
  * the paper's Theorem (Section 2, after mam 2) on random convex chains.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1203_5004_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_hand_cases():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "hand_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, *rest = line.split()
            if tag == "case":
                cur = {"name": rest[0]}
                cases.append(cur)
            elif tag == "pts":
                v = [int(t) for t in rest]
                cur["kx"] = np.array(v[0::2], dtype=np.int32)
                cur["ky"] = np.array(v[1::2], dtype=np.int32)
            elif tag == "hull":
                cur["hull"] = [int(t) for t in rest]
    return cases


HAND = load_hand_cases()


@pytest.mark.parametrize("case", HAND, ids=[c["name"] for c in HAND])
def test_hand_cases(case):
    assert oracle.upper_hull(case["kx"], case["ky"]).tolist() == case["hull"]
    assert oracle.upper_hull_brute(case["kx"], case["ky"]).tolist() == case["hull"]


def _small_sets():
    kinds = ["uniform", "arc", "band", "gauss_x", "gauss_disk", "columns", "duplicates"]
    out = []
    for kind in kinds:
        for n in (0, 1, 2, 3, 4, 5, 7, 8, 16, 31, 64, 100, 200):
            for seed in range(3):
                out.append((kind, n, seed))
    return out


@pytest.mark.parametrize("kind,n,seed", _small_sets())
def test_chain_equals_brute_force(kind, n, seed):
    ps = inputs.make(kind, n, 1000 + seed)
    a = oracle.upper_hull(ps.kx, ps.ky)
    b = oracle.upper_hull_brute(ps.kx, ps.ky)
    assert a.tolist() == b.tolist()


def test_brute_force_tiny_lattice_exhaustive():
    # Every sorted multiset of 4 points on a 3x3 lattice, which covers columns,
    # repeats, collinear triples and vertical edges at both ends.
    lattice = [(x, y) for x in range(3) for y in range(3)]
    rng = np.random.default_rng(0)
    for _ in range(3000):
        idx = np.sort(rng.integers(0, len(lattice), size=rng.integers(1, 7)))
        pts = [lattice[i] for i in idx]
        kx = np.array([p[0] for p in pts], np.int32)
        ky = np.array([p[1] for p in pts], np.int32)
        assert oracle.upper_hull(kx, ky).tolist() == oracle.upper_hull_brute(kx, ky).tolist()


def test_closed_form_concave_all_corners():
    ps = inputs.closed_form()
    h = oracle.upper_hull(ps.kx, ps.ky)
    assert h.tolist() == list(range(4096))


def test_closed_form_convex_only_ends():
    i = np.arange(4096, dtype=np.int64)
    kx, ky = (i << 12).astype(np.int32), (i * i).astype(np.int32)
    assert oracle.upper_hull(kx, ky).tolist() == [0, 4095]


def test_collinear_line_only_ends():
    i = np.arange(1000, dtype=np.int64)
    kx, ky = (i * 7 + 3).astype(np.int32), (i * 5 + 11).astype(np.int32)
    assert oracle.upper_hull(kx, ky).tolist() == [0, 999]


def test_single_column_only_ends():
    ky = np.arange(0, 5000, 3, dtype=np.int32)
    kx = np.full_like(ky, 12345)
    assert oracle.upper_hull(kx, ky).tolist() == [0, ky.shape[0] - 1]


def test_all_identical():
    kx = np.full(50, 9, np.int32)
    assert oracle.upper_hull(kx, kx).tolist() == [0]


def test_clamped_row_ends_only():
    # A Gaussian clipped at the top row y = 1 - 2^-24: many points on the same
    # horizontal line, which are collinear, so only the two ends are corners.
    r = np.random.default_rng(3)
    kx = np.sort(r.integers(0, inputs.G, 3000)).astype(np.int32)
    ky = np.full(3000, inputs.G - 1, np.int32)
    kx = np.unique(kx)
    ky = ky[: kx.shape[0]]
    assert oracle.upper_hull(kx, ky).tolist() == [0, kx.shape[0] - 1]


def _qhull_upper(kx, ky):
    from scipy.spatial import ConvexHull
    pts = np.stack([kx.astype(np.float64), ky.astype(np.float64)], axis=1)
    ccw = ConvexHull(pts).vertices.tolist()
    key = kx.astype(np.int64) * inputs.G + ky
    lo, hi = int(np.argmin(key)), int(np.argmax(key))
    k = ccw.index(hi)
    chain = []
    while True:
        chain.append(ccw[k])
        if ccw[k] == lo:
            break
        k = (k + 1) % len(ccw)
    return sorted(chain)


@pytest.mark.parametrize("n,seed", [(10, 1), (100, 2), (1000, 3), (20000, 4), (200000, 5)])
def test_matches_qhull_general_position(n, seed):
    pytest.importorskip("scipy")
    ps = inputs.uniform(n, seed)
    assert oracle.upper_hull(ps.kx, ps.ky).tolist() == _qhull_upper(ps.kx, ps.ky)


def _check_invariants(kx, ky, h):
    n = kx.shape[0]
    X, Y = kx.astype(np.int64), ky.astype(np.int64)
    key = X * inputs.G + Y
    assert h.shape[0] >= 1
    assert h[0] == 0
    assert np.all(np.diff(h) > 0)
    last = int(np.searchsorted(key, key[-1], side="left"))
    assert h[-1] == last
    hk = key[h]
    assert np.all(np.diff(hk) > 0)
    # every corner is the first occurrence of its coordinates
    first = np.searchsorted(key, hk, side="left")
    assert np.array_equal(first, h)
    # strict right turns at every interior corner
    if h.shape[0] >= 3:
        o, a, b = h[:-2], h[1:-1], h[2:]
        det = (X[a] - X[o]) * (Y[b] - Y[o]) - (Y[a] - Y[o]) * (X[b] - X[o])
        assert np.all(det < 0)
    # every input point lies on or below the chain (walk by lexicographic key)
    if h.shape[0] >= 2:
        e = np.searchsorted(hk, key, side="right") - 1
        e = np.clip(e, 0, h.shape[0] - 2)
        o, a = h[e], h[e + 1]
        det = (X[a] - X[o]) * (Y - Y[o]) - (Y[a] - Y[o]) * (X - X[o])
        assert np.all(det <= 0)
    else:
        assert np.all(key == key[0])


@pytest.mark.parametrize("kind", ["uniform", "arc", "band", "gauss_x", "gauss_disk", "columns", "duplicates"])
def test_invariants_large(kind):
    ps = inputs.make(kind, 300_000, 21)
    h = oracle.upper_hull(ps.kx, ps.ky)
    _check_invariants(ps.kx, ps.ky, h)


@pytest.mark.parametrize("kind", ["uniform", "arc", "band", "gauss_x", "duplicates"])
def test_hull_of_strip_hulls(kind):
    # The hull of a union is the hull of the union of the parts' hulls; this is
    # what every merge stage relies on (paper Section 3, strips).
    ps = inputs.make(kind, 100_000, 31)
    full = oracle.upper_hull(ps.kx, ps.ky)
    cuts = np.linspace(0, len(ps), 17).astype(np.int64)
    cand = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        cand.append(a + oracle.upper_hull(ps.kx[a:b], ps.ky[a:b]))
    cand = np.concatenate(cand)
    sub = oracle.upper_hull(ps.kx[cand], ps.ky[cand])
    merged = cand[sub]
    # A later repeat of a point may open a strip; map back to first occurrences.
    key = ps.kx.astype(np.int64) * inputs.G + ps.ky
    merged = np.searchsorted(key, key[merged], side="left")
    assert merged.tolist() == full.tolist()


def test_orient_sign_big_integers():
    r = np.random.default_rng(9)
    pts = r.integers(0, inputs.G, size=(30000, 2)).astype(np.int32)
    # add extreme and collinear triples
    ext = np.array([[0, 0], [inputs.G - 1, inputs.G - 1], [inputs.G - 1, 0],
                    [0, 0], [1, 1], [2, 2],
                    [0, inputs.G - 1], [inputs.G - 1, 0], [1, inputs.G - 2]], np.int32)
    pts = np.concatenate([pts, ext])
    s = oracle.orient_signs(pts[:, 0], pts[:, 1])
    for t in range(s.shape[0]):
        (ox, oy), (ax, ay), (bx, by) = (tuple(int(v) for v in pts[3 * t + i]) for i in range(3))
        d = (ax - ox) * (by - oy) - (ay - oy) * (bx - ox)
        assert s[t] == (d > 0) - (d < 0)


def _random_hood(r, n, x0, x1):
    """Upper hood of n random grid points with x in [x0, x1)."""
    kx = r.integers(x0, x1, size=n)
    ky = r.integers(0, inputs.G, size=n)
    kx, ky = inputs.sort_lex(kx, ky)
    h = oracle.upper_hull(kx, ky)
    return kx[h].astype(np.int64), ky[h].astype(np.int64)


def _orient(o, a, b):
    return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])


def test_bridge_is_supporting_line():
    # The bridge from the merged hood equals the brute-force supporting line:
    # all of P and Q on or below line(P[p], Q[q]); leftmost such P corner and
    # rightmost such Q corner.
    r = np.random.default_rng(5)
    for trial in range(300):
        hp, hq = int(r.integers(1, 40)), int(r.integers(1, 40))
        split = int(r.integers(1 << 10, inputs.G - (1 << 10)))
        px, py = _random_hood(r, hp, 0, split)
        qx, qy = _random_hood(r, hq, split, inputs.G)
        p, q = oracle.bridge(px, py, qx, qy)
        pts = list(zip(px.tolist(), py.tolist())) + list(zip(qx.tolist(), qy.tolist()))
        cands = []
        for i in range(len(px)):
            for j in range(len(qx)):
                a, b = (int(px[i]), int(py[i])), (int(qx[j]), int(qy[j]))
                if all(_orient(a, b, c) <= 0 for c in pts):
                    cands.append((i, j))
        best_p = min(i for i, _ in cands)
        best_q = max(j for i, j in cands if i == best_p)
        assert (p, q) == (best_p, best_q), trial


def test_theorem_tangent_monotone():
    # Paper Section 2, Theorem: the tangent corners q'_i of H(Q) seen from the
    # corners p_i of H(P) are non-decreasing left to right, and p_i is left of,
    # at, or right of the bridge corner p as f(p_i, q'_i) is LOW, EQUAL, HIGH.
    r = np.random.default_rng(6)
    for trial in range(300):
        hp, hq = int(r.integers(1, 30)), int(r.integers(1, 30))
        split = int(r.integers(1 << 10, inputs.G - (1 << 10)))
        px, py = _random_hood(r, hp, 0, split)
        qx, qy = _random_hood(r, hq, split, inputs.G)
        P = list(zip(px.tolist(), py.tolist()))
        Q = list(zip(qx.tolist(), qy.tolist()))

        def tangent(pt):
            # rightmost corner of Q on the supporting line from pt
            for j in range(len(Q) - 1, -1, -1):
                if all(_orient(pt, Q[j], c) <= 0 for c in Q):
                    return j
            raise AssertionError

        def f(i, j):
            # where P[i] sits relative to the leftmost tangent corner of H(P) from Q[j]
            for k in range(len(P)):
                if all(_orient(P[k], Q[j], c) <= 0 for c in P):
                    t = k
                    break
            return (i > t) - (i < t)

        tq = [tangent(p) for p in P]
        fs = [f(i, tq[i]) for i in range(len(P))]
        bp, bq = oracle.bridge(px, py, qx, qy)
        # The classification holds for every corner of H(P) ...
        assert fs == [(-1 if i < bp else (0 if i == bp else 1)) for i in range(len(P))], trial
        # ... but the monotone order of tangent corners only up to the bridge
        # corner (see test_theorem_monotonicity_counterexample).
        assert all(a <= b for a, b in zip(tq[:bp + 1], tq[1:bp + 1])), trial
        assert tq[bp] == bq


def test_theorem_monotonicity_counterexample():
    # The Theorem's first claim fails to the right of the bridge corner: from
    # P = (0,0),(5,100),(9,0) the tangent corners on Q = (10,0),(11,10),(12,0)
    # are 1, 2, 1. The LOW/EQUAL/HIGH classification still holds, and that is
    # the only part the bridge search uses.
    P = [(0, 0), (5, 100), (9, 0)]
    Q = [(10, 0), (11, 10), (12, 0)]

    def tangent(pt):
        for j in range(len(Q) - 1, -1, -1):
            if all(_orient(pt, Q[j], c) <= 0 for c in Q):
                return j

    assert [tangent(p) for p in P] == [1, 2, 1]
    px, py = zip(*P)
    qx, qy = zip(*Q)
    assert oracle.bridge(px, py, qx, qy) == (1, 2)


def test_batched_matches_per_set():
    ps, offs, _ = inputs.batched(200, seed=8, hi=3000)
    out, counts = oracle.upper_hull_batched(ps.kx, ps.ky, offs)
    for s in range(200):
        a, b = offs[s], offs[s + 1]
        ref = oracle.upper_hull(ps.kx[a:b], ps.ky[a:b])
        assert out[a:a + counts[s]].tolist() == ref.tolist()


# ---------------------------------------------------------------- strip-parallel baseline
@pytest.mark.parametrize("kind", ["uniform", "arc", "band", "gauss_x", "gauss_disk", "columns", "duplicates"])
def test_strips_equal_chain(kind):
    # The strip-parallel run (the CPU baseline) must give the single scan's
    # index list for every strip count, including strips that cut through
    # runs of repeats and columns, and strips of one or two points.
    for n in (0, 1, 2, 3, 4, 9, 33, 500, 4099, 70_001):
        ps = inputs.make(kind, n, 40 + n)
        ref = oracle.upper_hull(ps.kx, ps.ky)
        for t in (1, 2, 3, 5, 8, 16, 64):
            assert np.array_equal(oracle.upper_hull_strips(ps.kx, ps.ky, t), ref), (kind, n, t)


def test_strips_cut_inside_repeat_runs():
    # every strip boundary falls inside a long run of one repeated point, and
    # the chain's end points are repeats too
    kx = np.repeat(np.array([0, 5, 9, 14, 20], np.int32), 37)
    ky = np.repeat(np.array([3, 11, 12, 8, 1], np.int32), 37)
    ref = oracle.upper_hull_brute(kx, ky)
    assert ref.tolist() == [0, 37, 74, 111, 148]
    for t in range(1, 40):
        assert oracle.upper_hull_strips(kx, ky, t).tolist() == ref.tolist(), t


def test_strips_concave_closed_form():
    # every point of the closed-form concave sequence is a corner, whatever the strips
    ps = inputs.closed_form()
    for t in (2, 7, 16, 100):
        assert np.array_equal(oracle.upper_hull_strips(ps.kx, ps.ky, t), np.arange(4096))


def test_batched_threads_equal_batched():
    # the multi-threaded batched baseline gives the single-thread batched output
    ps, offs, _ = inputs.batched(700, seed=31, hi=3000)
    ref_out, ref_cnt = oracle.upper_hull_batched(ps.kx, ps.ky, offs)
    for t in (1, 2, 5, 16, 1000):
        out, cnt = oracle.upper_hull_batched_threads(ps.kx, ps.ky, offs, t)
        assert np.array_equal(cnt, ref_cnt), t
        for s in range(len(cnt)):
            a = offs[s]
            assert np.array_equal(out[a:a + cnt[s]], ref_out[a:a + cnt[s]]), (t, s)


# ---------------------------------------------------------------- lower hood and convex hull
@pytest.mark.parametrize("kind", ["uniform", "arc", "band", "gauss_x", "gauss_disk", "columns", "duplicates"])
def test_lower_chain_equals_brute_force(kind):
    for n in (0, 1, 2, 3, 4, 7, 16, 31, 100, 200):
        for seed in range(3):
            ps = inputs.make(kind, n, 300 + 7 * n + seed)
            assert np.array_equal(oracle.lower_hull(ps.kx, ps.ky), oracle.lower_hull_brute(ps.kx, ps.ky)), (kind, n)


def test_lower_chain_lattice_exhaustive():
    # every set of up to 5 distinct points on a 3 x 3 lattice, sorted
    import itertools
    pts = [(x, y) for x in range(3) for y in range(3)]
    for k in range(1, 6):
        for combo in itertools.combinations(pts, k):
            kx = np.array([p[0] for p in combo], np.int32)
            ky = np.array([p[1] for p in combo], np.int32)
            assert np.array_equal(oracle.lower_hull(kx, ky), oracle.lower_hull_brute(kx, ky)), combo


def test_lower_chain_is_mirrored_upper_chain_distinct_x():
    # with distinct x values, mirroring y (ky -> G - 1 - ky) keeps the order,
    # and the lower hood is the mirror image of the upper hood
    r = np.random.default_rng(5)
    for n in (3, 10, 100, 5000):
        kx = np.sort(r.choice(inputs.G, size=n, replace=False)).astype(np.int32)
        ky = r.integers(0, inputs.G, size=n).astype(np.int32)
        assert np.array_equal(oracle.lower_hull(kx, ky), oracle.upper_hull(kx, inputs.G - 1 - ky))


def test_lower_chain_closed_forms():
    # an upward-convex parabola: every point is a lower corner, and the upper
    # hood has only the ends
    i = np.arange(2000, dtype=np.int64)
    kx = i * 4000
    ky = (i - 1000) ** 2 * 8
    assert np.array_equal(oracle.lower_hull(kx, ky), np.arange(2000))
    assert oracle.upper_hull(kx, ky).tolist() == [0, 1999]
    # a last column of several points: the lower hood ends with its vertical edge
    assert oracle.lower_hull([0, 5, 5, 5], [0, 1, 4, 9]).tolist() == [0, 1, 3]
    # repeats count once (first occurrence)
    assert oracle.lower_hull([0, 0, 3, 3, 6], [2, 2, 0, 0, 2]).tolist() == [0, 2, 4]


@pytest.mark.parametrize("n,seed", [(3, 1), (10, 2), (100, 3), (1000, 4), (20000, 5)])
def test_convex_hull_matches_qhull_general_position(n, seed):
    spatial = pytest.importorskip("scipy.spatial")
    r = np.random.default_rng(seed)
    kx = r.choice(inputs.G, size=n, replace=False)
    ky = r.choice(inputs.G, size=n, replace=False)
    kx, ky = inputs.sort_lex(kx, ky)
    got = oracle.convex_hull(kx, ky)
    ref = spatial.ConvexHull(np.stack([kx, ky], 1).astype(np.float64)).vertices
    assert sorted(got.tolist()) == sorted(ref.tolist())
    assert got[0] == 0 and len(set(got.tolist())) == len(got)
    # clockwise: negative signed area
    x = kx[got].astype(np.float64)
    y = ky[got].astype(np.float64)
    assert np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y) < 0


@pytest.mark.parametrize("kind", ["uniform", "arc", "band", "gauss_x", "columns", "duplicates"])
def test_convex_hull_is_upper_then_lower_brute(kind):
    # the stitched hull equals the brute-force upper corners followed by the
    # brute-force lower corners, reversed, without the shared ends
    for n in (1, 2, 3, 5, 40, 150):
        ps = inputs.make(kind, n, 900 + n)
        up = oracle.upper_hull_brute(ps.kx, ps.ky).tolist()
        lo = oracle.lower_hull_brute(ps.kx, ps.ky).tolist()
        assert oracle.convex_hull(ps.kx, ps.ky).tolist() == up + lo[::-1][1:-1], (kind, n)


def test_convex_hull_degenerate():
    assert oracle.convex_hull([], []).tolist() == []
    assert oracle.convex_hull([7], [7]).tolist() == [0]
    assert oracle.convex_hull([7, 7, 7], [7, 7, 7]).tolist() == [0]
    assert oracle.convex_hull([0, 1, 2, 3], [0, 1, 2, 3]).tolist() == [0, 3]  # collinear
    assert oracle.convex_hull([0, 0, 0], [0, 1, 2]).tolist() == [0, 2]  # one column
    # a square with its centre and a point on an edge
    kx = [0, 0, 1, 2, 2, 2]
    ky = [0, 2, 1, 0, 1, 2]
    assert oracle.convex_hull(kx, ky).tolist() == [0, 1, 5, 3]


# ---------------------------------------------------------------- sort (the step before the path)
@pytest.mark.parametrize("n,seed", [(0, 0), (1, 1), (2, 2), (50, 3), (1000, 4), (5000, 5)])
def test_sort_points_matches_python_sorted(n, seed):
    # Python's sort is stable and compares the (x, y) pairs themselves: an
    # independent statement of the same order
    r = np.random.default_rng(seed)
    kx = r.integers(0, 8, size=n)        # few distinct x: ties in x
    ky = r.integers(0, 1 << 24, size=n)
    ky[r.random(n) < 0.3] = 5            # repeated points
    got = oracle.sort_points(kx, ky)
    want = sorted(range(n), key=lambda i: (int(kx[i]), int(ky[i])))
    assert got.tolist() == want


def test_sort_points_invariants():
    r = np.random.default_rng(9)
    kx = r.integers(0, 1 << 24, size=20_000)
    ky = r.integers(0, 1 << 24, size=20_000)
    kx[::7] = kx[0]
    ky[::11] = ky[3]
    perm = oracle.sort_points(kx, ky)
    assert sorted(perm.tolist()) == list(range(kx.size))              # a permutation
    a, b = kx[perm], ky[perm]
    assert np.all((a[1:] > a[:-1]) | ((a[1:] == a[:-1]) & (b[1:] >= b[:-1])))  # sorted by (x, y)
    same = (a[1:] == a[:-1]) & (b[1:] == b[:-1])
    assert np.all(perm[1:][same] > perm[:-1][same])                  # stable


def test_sort_points_planted_unstable_sort_fails():
    # an unstable sort of the same keys is a plausible slip; the pin above
    # must tell it apart on repeated points
    kx = np.array([3, 1, 3, 1, 3] * 40)
    ky = np.array([2, 9, 2, 9, 2] * 40)
    unstable = np.argsort((kx.astype(np.int64) << 24) | ky, kind="quicksort")[::-1]
    unstable = unstable[np.argsort((kx[unstable].astype(np.int64) << 24) | ky[unstable], kind="stable")]
    want = sorted(range(kx.size), key=lambda i: (int(kx[i]), int(ky[i])))
    assert unstable.tolist() != want
    assert oracle.sort_points(kx, ky).tolist() == want
