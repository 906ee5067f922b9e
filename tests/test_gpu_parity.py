"""GPU parity: every path through the C ABI against the CPU oracle, element by
element (corner index lists must be identical; the path is exact)."""
import numpy as np
import pytest

import oracle
from paper_1203_5004_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def wg():
    import __graft_entry__ as g
    g.build_library()
    from paper_1203_5004_gb300 import wagener
    wagener.load()
    return wagener


DEV = "cuda"
TILE_POINTS = {1: 128 * 31, 2: 128 * 23, 3: 256 * 31, 4: 256 * 15}


def gpu_points(ps):
    return torch.from_numpy(ps.points()).to(DEV)


def assert_same(got, ref, what=""):
    got = np.asarray(got)
    if not np.array_equal(got, ref):
        n = min(len(got), len(ref))
        bad = np.nonzero(got[:n] != ref[:n])[0]
        first = int(bad[0]) if bad.size else n
        raise AssertionError(f"{what}: {len(got)} vs {len(ref)} corners, first difference at {first}: "
                             f"gpu {got[first:first + 5].tolist()} oracle {ref[first:first + 5].tolist()}")


# ---------------------------------------------------------------- predicate
def _near_collinear(r, n):
    o = r.integers(0, inputs.G // 2, size=(n, 2))
    d = r.integers(-(1 << 10), 1 << 10, size=(n, 2))
    k = r.integers(1, 1 << 10, size=(n, 1))
    m = r.integers(1, 1 << 10, size=(n, 1))
    eps = r.integers(-1, 2, size=(n, 2))
    a = o + k * d
    b = o + m * d + eps
    pts = np.stack([o, a, b], axis=1).reshape(-1, 2)
    return np.clip(pts, 0, inputs.G - 1).astype(np.int32)


@pytest.mark.parametrize("mode", [0, 1])
def test_orient_signs(wg, mode):
    r = np.random.default_rng(1)
    rand = r.integers(0, inputs.G, size=(3 * 200_000, 2)).astype(np.int32)
    near = _near_collinear(r, 200_000)
    # thin tiles: all three points within a few grid units of a long line
    pts = np.concatenate([rand, near])
    ref = oracle.orient_signs(pts[:, 0], pts[:, 1])
    t = torch.from_numpy(inputs.to_float_points(pts[:, 0], pts[:, 1])).to(DEV)
    signs, fb = wg.debug_orient(t, pred_mode=mode)
    assert_same(signs.cpu().numpy(), ref, "orient signs")
    if mode == 0:
        assert fb > 0  # the near-collinear triples must reach the float64 path
        assert fb < ref.shape[0]


def test_orient_small_differences_exact_without_fallback(wg):
    # All three points within 2^11 grid units of each other: both products are
    # below 2^23 units of 2^-48, so the float32 determinant is exact (zero
    # included) and no triple needs the float64 path.
    r = np.random.default_rng(3)
    n = 300_000
    o = r.integers(0, inputs.G - (1 << 11), size=(n, 1, 2))
    off = r.integers(0, 1 << 11, size=(n, 3, 2))
    # every third triple exactly collinear: c, c + d, c + m d with m in {0, 1, 2}
    d = r.integers(-(1 << 5), 1 << 5, size=(n, 2))
    m = r.integers(0, 3, size=(n, 1))
    c = np.full_like(d, 1 << 10)
    col = np.stack([c, c + d, c + m * d], axis=1)
    pts = np.where((np.arange(n) % 3 == 0)[:, None, None], col, off) + o
    pts = np.clip(pts.reshape(-1, 2), 0, inputs.G - 1).astype(np.int32)
    ref = oracle.orient_signs(pts[:, 0], pts[:, 1])
    assert (ref == 0).sum() > n // 4
    t = torch.from_numpy(inputs.to_float_points(pts[:, 0], pts[:, 1])).to(DEV)
    signs, fb = wg.debug_orient(t, pred_mode=0)
    assert_same(signs.cpu().numpy(), ref, "orient signs, small differences")
    assert fb == 0


# ---------------------------------------------------------------- bridge
def _hood_pair(r, n, span, kind):
    if kind == "concave":
        # a strictly concave integer chain (every point a hood corner), some
        # points pushed down: long hoods, bridges anywhere along them
        i = np.arange(n, dtype=np.int64)
        d = int(r.integers(1, 64))
        kx = int(r.integers(0, inputs.G // 2)) + i * d
        ky = (1 << 20) + i * (n - i) * int(r.integers(1, 8))
        ky = ky - (r.random(n) < 0.2) * r.integers(0, 1 << 12, size=n)
    elif kind == "arc":
        # points on the quantised parabola of the arc workload, in a narrow x
        # window: long runs of hood corners, near-collinear triples
        x0 = int(r.integers(0, inputs.G - (1 << 16)))
        kx = x0 + r.integers(0, 1 << int(r.integers(6, 16)), size=n)
        ky = inputs._arc_ky(kx)
    else:
        kx = r.integers(0, span, size=n) * (inputs.G // span if kind == "coarse" else 1)
        ky = r.integers(0, inputs.G, size=n) if kind != "coarse" else r.integers(0, span, size=n) * (inputs.G // span)
    kx, ky = inputs.sort_lex(kx, ky)
    key = kx.astype(np.int64) * inputs.G + ky
    _, first = np.unique(key, return_index=True)
    kx, ky = kx[first], ky[first]
    if kx.shape[0] < 2:
        return None
    k = int(r.integers(1, kx.shape[0]))
    hp = oracle.upper_hull(kx[:k], ky[:k])
    hq = oracle.upper_hull(kx[k:], ky[k:]) + k
    return kx, ky, hp, hq


@pytest.mark.parametrize("kind", ["fine", "coarse", "arc", "concave"])
def test_bridge_against_oracle(wg, kind):
    r = np.random.default_rng({"fine": 2, "coarse": 3, "arc": 13, "concave": 14}[kind])
    checked = 0
    for trial in range(400):
        n = int(r.integers(2, {"arc": 400, "concave": 600}.get(kind, 3000)))
        span = int(r.integers(2, 64)) if kind == "coarse" else inputs.G
        pair = _hood_pair(r, n, span, kind)
        if pair is None:
            continue
        kx, ky, hp, hq = pair
        ref = oracle.bridge(kx[hp], ky[hp], kx[hq], ky[hq])
        P = torch.from_numpy(inputs.to_float_points(kx[hp], ky[hp])).to(DEV)
        Q = torch.from_numpy(inputs.to_float_points(kx[hq], ky[hq])).to(DEV)
        got = wg.debug_bridge(P, Q)
        assert got == ref, (trial, got, ref, len(hp), len(hq))
        checked += 1
    assert checked > 300


def test_warp_hood_against_oracle(wg):
    r = np.random.default_rng(4)
    for trial in range(1500):
        m = int(r.integers(0, 33))
        span = int(r.choice([4, 16, 1 << 12, inputs.G]))
        kx = r.integers(0, span, size=m) * (inputs.G // span)
        ky = r.integers(0, span, size=m) * (inputs.G // span)
        kx, ky = inputs.sort_lex(kx, ky)
        key = kx.astype(np.int64) * inputs.G + ky
        _, first = np.unique(key, return_index=True)
        kx, ky = kx[first], ky[first]
        ref = oracle.upper_hull(kx, ky)
        t = torch.from_numpy(inputs.to_float_points(kx, ky)).to(DEV) if kx.shape[0] else \
            torch.empty((0, 2), dtype=torch.float32, device=DEV)
        got = wg.debug_warp_hood(t)
        assert_same(got, ref, f"warp hood trial {trial}")


# ---------------------------------------------------------------- whole path
KINDS = ["uniform", "arc", "band", "gauss_x", "columns", "duplicates"]


@pytest.mark.parametrize("kind", KINDS)
def test_small_n_sweep(wg, kind):
    ws = wg.new_workspace(wg.workspace_size(1000))
    for n in range(0, 301):
        ps = inputs.make(kind, n, 100 + n)
        got = wg.upper_hood(gpu_points(ps), workspace=ws).cpu().numpy() if n else \
            wg.upper_hood(torch.empty((0, 2), dtype=torch.float32, device=DEV), workspace=ws).cpu().numpy()
        assert_same(got, oracle.upper_hull(ps.kx, ps.ky), f"{kind} n={n}")
    assert wg.device_status(ws) == 0


@pytest.mark.parametrize("cfg", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", KINDS)
def test_tile_edges(wg, cfg, kind):
    T = TILE_POINTS[cfg]
    opts = wg.default_options(tile_config=cfg)
    ws = wg.new_workspace(wg.workspace_size(1 << 22))
    for n in (T - 1, T, T + 1, 2 * T - 1, 3 * T + 7, 17 * T + 5, 200 * T + 3):
        ps = inputs.make(kind, n, n)
        got = wg.upper_hood(gpu_points(ps), opts=opts, workspace=ws).cpu().numpy()
        assert_same(got, oracle.upper_hull(ps.kx, ps.ky), f"cfg{cfg} {kind} n={n}")
    assert wg.device_status(ws) == 0


@pytest.mark.parametrize("k", list(range(1, 22)))
def test_powers_of_two(wg, k):
    for n in (2 ** k - 1, 2 ** k, 2 ** k + 1):
        ps = inputs.uniform(n, k)
        got = wg.upper_hood(gpu_points(ps)).cpu().numpy()
        assert_same(got, oracle.upper_hull(ps.kx, ps.ky), f"uniform n={n}")


@pytest.mark.parametrize("spc", [1, 2, 4, 8])
def test_segments_per_cta(wg, spc):
    ps = inputs.band(3_000_000, 9)
    ref = oracle.upper_hull(ps.kx, ps.ky)
    for cfg in (1, 2, 3, 4):
        got = wg.upper_hood(gpu_points(ps), opts=wg.default_options(tile_config=cfg, segments_per_cta=spc))
        assert_same(got.cpu().numpy(), ref, f"cfg{cfg} spc{spc}")


def _tall_columns(seed, first, mid, last, rest, rep_every):
    """Sorted points with three tall columns: the set's first column (every
    point a new height maximum), one in the middle and the last one; every
    rep_every-th point of each column repeated, so that repeats fall on tile
    edges somewhere; `rest` uniform points between them."""
    r = np.random.default_rng(seed)
    G = inputs.G
    cols = []
    for x, m in ((0, first), (G // 2 + 17, mid), (G - 1, last)):
        ys = np.sort(r.choice(G, size=m, replace=False)).astype(np.int64)
        ys = np.concatenate([ys, ys[::rep_every]])
        cols.append((np.full(ys.shape, x, np.int64), ys))
    kx = np.concatenate([c[0] for c in cols] + [r.integers(1, G - 1, size=rest)])
    ky = np.concatenate([c[1] for c in cols] + [r.integers(0, G, size=rest)])
    return inputs.PointSet(*inputs.sort_lex(kx, ky), name="tall_columns")


@pytest.mark.parametrize("cfg", [1, 2, 3, 4])
def test_tall_columns(wg, cfg):
    # Tiles that lie in one column take their own path (the column rule over
    # the strip, no height rule): the first column, where the height rule
    # drops nothing, a middle column and the last one, with repeats.
    T = TILE_POINTS[cfg]
    opts = wg.default_options(tile_config=cfg)
    for seed, (first, mid, last, rest, rep) in enumerate([
            (7 * T + 3, 3 * T + 1, 2 * T - 1, 20000, 31),
            (T - 1, T + 1, T, 5000, 7),
            (40 * T + 11, 0 + 1, 9 * T, 300000, 97),
            (3 * T, 5 * T, 3 * T, 0, 2)]):
        ps = _tall_columns(seed, first, mid, last, rest, rep)
        got = wg.upper_hood(gpu_points(ps), opts=opts).cpu().numpy()
        assert_same(got, oracle.upper_hull(ps.kx, ps.ky), f"cfg{cfg} tall columns seed {seed}")


SMALL_SIZES = (1, 2, 3, 15, 16, 17, 31, 33, 511, 512, 513, 4095, 4096, 4097, 8191, 8192)


@pytest.mark.parametrize("kind", KINDS + ["gauss_disk"])
def test_small_path(wg, kind):
    # One CTA, 16 points per thread: sizes around the thread and warp edges
    # up to the path's limit, both as the default and when forced.
    ws = wg.new_workspace(wg.workspace_size(8192))
    forced = wg.default_options(schedule=4)
    for n in SMALL_SIZES:
        ps = inputs.make(kind, n, n + 3)
        ref = oracle.upper_hull(ps.kx, ps.ky)
        assert_same(wg.upper_hood(gpu_points(ps), workspace=ws).cpu().numpy(), ref, f"{kind} n={n}")
        assert_same(wg.upper_hood(gpu_points(ps), opts=forced, workspace=ws).cpu().numpy(), ref,
                    f"{kind} n={n} forced")
    assert wg.device_status(ws) == 0


def test_small_path_modes_and_views(wg):
    # float64-only predicate, counters, validation, an unaligned view and the
    # closed form (every point a corner: the list stays whole)
    ws = wg.new_workspace(wg.workspace_size(8192))
    for kind in ("band", "arc", "duplicates"):
        ps = inputs.make(kind, 8001, 11)
        ref = oracle.upper_hull(ps.kx, ps.ky)
        for o in (wg.default_options(pred_mode=1), wg.default_options(count_predicates=1),
                  wg.default_options(validate=1)):
            assert_same(wg.upper_hood(gpu_points(ps), opts=o, workspace=ws).cpu().numpy(), ref, f"{kind} modes")
        base = torch.zeros((len(ps) + 1, 2), dtype=torch.float32, device=DEV)
        base[1:] = gpu_points(ps)
        assert base[1:].data_ptr() % 16 == 8
        assert_same(wg.upper_hood(base[1:], workspace=ws).cpu().numpy(), ref, f"{kind} unaligned")
    assert wg.device_status(ws) == 0
    tests, _ = wg.read_counters(ws)
    assert tests > 0
    ps = inputs.closed_form()
    got = wg.upper_hood(gpu_points(ps), opts=wg.default_options(schedule=4), workspace=ws).cpu().numpy()
    assert_same(got, np.arange(4096, dtype=np.int32), "closed form, small path")


def test_small_path_validation_and_limit(wg):
    ps = inputs.uniform(8000, 5)
    pts = gpu_points(ps)
    ws = wg.new_workspace(wg.workspace_size(len(ps)))
    o = wg.default_options(validate=1, schedule=4)
    out = torch.empty(len(ps), dtype=torch.int32, device=DEV)
    cnt = torch.empty(1, dtype=torch.int32, device=DEV)
    bad = pts.clone()
    bad[[4095, 4096]] = bad[[4096, 4095]]  # across a thread (and warp) edge
    wg.upper_hood_into(bad, out, cnt, ws, o)
    assert wg.device_status(ws) == 3
    bad = pts.clone()
    bad[5000, 1] = float(np.float32(0.3) + np.float32(2.0 ** -25))
    wg.upper_hood_into(bad, out, cnt, ws, o)
    assert wg.device_status(ws) == 4
    big = inputs.uniform(8193, 1)
    with pytest.raises(wg.WagenerError):
        wg.upper_hood(gpu_points(big), opts=wg.default_options(schedule=4))


def test_closed_form_all_corners(wg):
    ps = inputs.closed_form()
    got = wg.upper_hood(gpu_points(ps)).cpu().numpy()
    assert_same(got, np.arange(4096, dtype=np.int32), "closed form")


def test_unaligned_points(wg):
    # a view that starts 8 bytes past a 16-byte boundary: every tile is staged
    # with a one-point shift
    for kind in ("uniform", "band", "duplicates"):
        ps = inputs.make(kind, 1_000_001, 5)
        base = torch.zeros((len(ps) + 1, 2), dtype=torch.float32, device=DEV)
        base[1:] = gpu_points(ps)
        view = base[1:]
        assert view.data_ptr() % 16 == 8
        got = wg.upper_hood(view).cpu().numpy()
        assert_same(got, oracle.upper_hull(ps.kx, ps.ky), f"unaligned {kind}")


def test_long_hood_spills_window(wg):
    # Every point of a long strictly concave chain is a corner: the running
    # hood outgrows its shared window and spills to the output array.
    # y = i (N - i) / 2 (exact: N is odd) has second difference -1: every
    # point is a corner.
    N = 11583
    i = np.arange(N + 1, dtype=np.int64)
    kx = i * 1448
    ky = i * (N - i) // 2
    ps = inputs.PointSet(kx, ky)
    ref = oracle.upper_hull(ps.kx, ps.ky)
    assert ref.shape[0] == N + 1
    for cfg in (1, 2, 3, 4):
        got = wg.upper_hood(gpu_points(ps), opts=wg.default_options(tile_config=cfg)).cpu().numpy()
        assert_same(got, ref, f"concave chain cfg{cfg}")


@pytest.mark.parametrize("name,make", [
    ("2^16 uniform", lambda: inputs.uniform(1 << 16, 1)),
    ("2^24 uniform", lambda: inputs.uniform(1 << 24, 2)),
    ("2^24 arc", lambda: inputs.arc(1 << 24, 3)),
    ("2^26 uniform", lambda: inputs.uniform(1 << 26, 7)),
])
def test_configs(wg, name, make):
    ps = make()
    ref = oracle.upper_hull(ps.kx, ps.ky)
    got = wg.upper_hood(gpu_points(ps)).cpu().numpy()
    assert_same(got, ref, name)


_FULL = {}


def _full(name):
    # the bench's full-size workloads, each generated and solved by the
    # oracle once per test session
    if name not in _FULL:
        ps = {"uniform26": lambda: inputs.uniform(1 << 26, 7), "band26": lambda: inputs.band(1 << 26, 4),
              "arc24": lambda: inputs.arc(1 << 24, 3)}[name]()
        _FULL[name] = (ps, oracle.upper_hull(ps.kx, ps.ky))
    return _FULL[name]


@pytest.mark.parametrize("name", ["uniform26", "band26", "arc24"])
@pytest.mark.parametrize("cfg,spc", [(1, 1), (2, 1), (2, 2), (3, 1), (3, 2), (4, 1)])
def test_full_size_every_launch_configuration(wg, name, cfg, spc):
    # every tile configuration and segment count the autotuner may pick for
    # the bench's workloads, at their full sizes
    ps, ref = _full(name)
    got = wg.upper_hood(gpu_points(ps), opts=wg.default_options(tile_config=cfg, segments_per_cta=spc))
    assert_same(got.cpu().numpy(), ref, f"{name} cfg{cfg} spc{spc}")


@pytest.mark.parametrize("name", ["uniform26", "band26"])
def test_full_size_autotuned_as_benched(wg, name):
    # the launch bench.py times: the autotuner's choice, then calls on one
    # workspace back to back
    ps, ref = _full(name)
    pts = gpu_points(ps)
    ws = wg.new_workspace(wg.workspace_size(len(ps)))
    best = wg.autotune(pts, ws)
    out = torch.empty(len(ps), dtype=torch.int32, device=DEV)
    cnt = torch.empty(1, dtype=torch.int32, device=DEV)
    for _ in range(3):
        wg.upper_hood_into(pts, out, cnt, ws, best)
    torch.cuda.synchronize()
    assert_same(out[: int(cnt.item())].cpu().numpy(), ref, f"{name} autotuned")
    assert wg.device_status(ws) == 0


def test_band_2_26_filtered_and_fp64(wg):
    ps = inputs.band(1 << 26, 4)
    ref = oracle.upper_hull(ps.kx, ps.ky)
    pts = gpu_points(ps)
    ws = wg.new_workspace(wg.workspace_size(len(ps)))
    for mode in (0, 1):
        o = wg.default_options(pred_mode=mode, count_predicates=1)
        out = torch.empty(len(ps), dtype=torch.int32, device=DEV)
        cnt = torch.empty(1, dtype=torch.int32, device=DEV)
        wg.upper_hood_into(pts, out, cnt, ws, o)
        got = out[: int(cnt.item())].cpu().numpy()
        assert_same(got, ref, f"band 2^26 mode {mode}")
        tests, fb = wg.read_counters(ws)
        assert tests > 0
        if mode == 0:
            assert 0 < fb < tests
        else:
            assert fb == 0
    assert wg.device_status(ws) == 0


@pytest.mark.slow
def test_gauss_x_2_28(wg):
    ps = inputs.gauss_x(1 << 28, 6)
    ref = oracle.upper_hull(ps.kx, ps.ky)
    pts = gpu_points(ps)
    del ps
    got = wg.upper_hood(pts).cpu().numpy()
    assert_same(got, ref, "gauss_x 2^28 fused")
    got = wg.upper_hood_plain(pts).cpu().numpy()
    assert_same(got, ref, "gauss_x 2^28 plain")


# ---------------------------------------------------------------- plain path
@pytest.mark.parametrize("kind", KINDS)
def test_plain_schedule(wg, kind):
    for n in (1, 2, 3, 5, 64, 1000, 4097, 100_003, 1 << 20):
        ps = inputs.make(kind, n, n + 1)
        got = wg.upper_hood_plain(gpu_points(ps)).cpu().numpy()
        assert_same(got, oracle.upper_hull(ps.kx, ps.ky), f"plain {kind} n={n}")


def test_plain_long_chain(wg):
    ps = inputs.closed_form()
    assert_same(wg.upper_hood_plain(gpu_points(ps)).cpu().numpy(), np.arange(4096, dtype=np.int32), "plain 2c")


# ---------------------------------------------------------------- batched
@pytest.mark.parametrize("num_sets,hi", [(1, 100), (50, 3000), (3000, 65536)])
def test_batched(wg, num_sets, hi):
    ps, offs, _ = inputs.batched(num_sets, seed=5 + num_sets, hi=hi)
    ref_out, ref_cnt = oracle.upper_hull_batched(ps.kx, ps.ky, offs)
    out, cnt = wg.upper_hood_batched(gpu_points(ps), offs)
    out, cnt = out.cpu().numpy(), cnt.cpu().numpy()
    assert_same(cnt, ref_cnt, "batched counts")
    for s in range(num_sets):
        a = offs[s]
        assert_same(out[a:a + cnt[s]], ref_out[a:a + ref_cnt[s]], f"set {s}")


def test_cuda_graph_replay(wg):
    # Both forms captured once in a CUDA graph and replayed: the workspace's
    # counters (arrivals, call counter, batched queue) reset themselves, so
    # every replay gives the oracle's corners.
    ps = inputs.make("band", 1 << 20, 21)
    ref = oracle.upper_hull(ps.kx, ps.ky)
    pts = gpu_points(ps)
    ws = wg.new_workspace(wg.workspace_size(len(ps)))
    out = torch.empty(len(ps), dtype=torch.int32, device=DEV)
    cnt = torch.empty(1, dtype=torch.int32, device=DEV)
    o = wg.default_options(tile_config=3)
    wg.upper_hood_into(pts, out, cnt, ws, o)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        wg.upper_hood_into(pts, out, cnt, ws, o)
    for _ in range(3):
        out.fill_(-1)
        cnt.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        assert_same(out[: int(cnt.item())].cpu().numpy(), ref, "single set, graph replay")
    assert wg.device_status(ws) == 0

    bps, offs, _ = inputs.batched(3000, seed=22)
    bref_out, bref_cnt = oracle.upper_hull_batched(bps.kx, bps.ky, offs)
    bpts = gpu_points(bps)
    offs_d = torch.from_numpy(offs).to(DEV)
    bout = torch.empty(max(int(offs[-1]), 1), dtype=torch.int32, device=DEV)
    bcnt = torch.empty(len(offs) - 1, dtype=torch.int32, device=DEV)
    bws = wg.new_workspace(wg.batched_workspace_size(offs))
    wg.upper_hood_batched_into(bpts, offs_d, bout, bcnt, bws)
    torch.cuda.synchronize()
    bg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(bg):
        wg.upper_hood_batched_into(bpts, offs_d, bout, bcnt, bws)
    for _ in range(3):
        bout.fill_(-1)
        bcnt.fill_(-1)
        bg.replay()
        torch.cuda.synchronize()
        c = bcnt.cpu().numpy()
        assert_same(c, bref_cnt, "batched counts, graph replay")
        o_ = bout.cpu().numpy()
        for s_ in range(0, len(offs) - 1, 97):
            a = int(offs[s_])
            assert_same(o_[a:a + c[s_]], bref_out[a:a + bref_cnt[s_]], f"batched set {s_}, graph replay")
    assert wg.device_status(bws) == 0


@pytest.mark.slow
def test_batched_full_100k(wg):
    # the batched workload at its full size (100,000 sets), every set checked
    ps, offs, _ = inputs.batched(100_000, seed=5)
    ref_out, ref_cnt = oracle.upper_hull_batched(ps.kx, ps.ky, offs)
    out, cnt = wg.upper_hood_batched(gpu_points(ps), offs)
    out, cnt = out.cpu().numpy(), cnt.cpu().numpy()
    assert_same(cnt, ref_cnt, "batched counts")
    # corners: compare the CSR-aligned arrays on every set's valid prefix at once
    n = offs[-1]
    valid = np.zeros(n, dtype=bool)
    starts = offs[:-1]
    for s in np.nonzero(ref_cnt)[0]:
        valid[starts[s]:starts[s] + ref_cnt[s]] = True
    assert np.array_equal(out[:n][valid], ref_out[:n][valid])


@pytest.mark.slow
def test_batched_full_100k_autotuned(wg):
    # the batched workload at its full size through the autotuned launch the
    # bench times (tile configuration and segment cap chosen on these sets),
    # every set checked against the oracle
    ps, offs, _ = inputs.batched(100_000, seed=5)
    ref_out, ref_cnt = oracle.upper_hull_batched(ps.kx, ps.ky, offs)
    pts = gpu_points(ps)
    offs_d = torch.from_numpy(offs).to(DEV)
    ws = wg.new_workspace(wg.batched_workspace_size(offs))
    best = wg.autotune_batched(pts, offs_d, ws)
    assert 1 <= best.tile_config <= 4 and best.batch_seg_tiles in (16, 32, 128)
    n = int(offs[-1])
    out = torch.empty(n, dtype=torch.int32, device=DEV)
    cnt = torch.empty(len(offs) - 1, dtype=torch.int32, device=DEV)
    for _ in range(2):
        wg.upper_hood_batched_into(pts, offs_d, out, cnt, ws, best)
    out, cnt = out.cpu().numpy(), cnt.cpu().numpy()
    assert_same(cnt, ref_cnt, "batched counts, autotuned")
    valid = np.zeros(n, dtype=bool)
    for s in np.nonzero(ref_cnt)[0]:
        valid[offs[s]:offs[s] + ref_cnt[s]] = True
    assert np.array_equal(out[valid], ref_out[:n][valid])
    assert wg.device_status(ws) == 0


@pytest.mark.parametrize("cap", [8, 16, 32])
def test_batched_split_sets(wg, cap):
    # small segment caps split the larger sets over several warps
    ps, offs, _ = inputs.batched(2000, seed=41, hi=65536)
    ref_out, ref_cnt = oracle.upper_hull_batched(ps.kx, ps.ky, offs)
    for cfg in (2, 3):
        out, cnt = wg.upper_hood_batched(gpu_points(ps), offs, wg.default_options(tile_config=cfg, batch_seg_tiles=cap))
        out, cnt = out.cpu().numpy(), cnt.cpu().numpy()
        assert_same(cnt, ref_cnt, f"batched counts cap {cap} cfg {cfg}")
        for s in range(len(cnt)):
            a = offs[s]
            assert_same(out[a:a + cnt[s]], ref_out[a:a + ref_cnt[s]], f"set {s} cap {cap} cfg {cfg}")


def test_batched_with_empty_and_large_sets(wg):
    sizes = [0, 1, 2, 0, 5, 300_000, 0, 7, 1_000_000, 3]
    sets = [inputs.make(k, n, i) for i, (k, n) in enumerate(zip(
        ["uniform", "band", "arc", "uniform", "duplicates", "band", "arc", "columns", "gauss_x", "uniform"], sizes))]
    kx = np.concatenate([s.kx for s in sets])
    ky = np.concatenate([s.ky for s in sets])
    offs = np.zeros(len(sizes) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    ref_out, ref_cnt = oracle.upper_hull_batched(kx, ky, offs)
    pts = torch.from_numpy(inputs.to_float_points(kx, ky)).to(DEV)
    for rep in range(2):
        out, cnt = wg.upper_hood_batched(pts, offs)
        out, cnt = out.cpu().numpy(), cnt.cpu().numpy()
        assert_same(cnt, ref_cnt, "counts")
        for s in range(len(sizes)):
            a = offs[s]
            assert_same(out[a:a + cnt[s]], ref_out[a:a + ref_cnt[s]], f"set {s}")


# ---------------------------------------------------------------- options
def test_validation_reports(wg):
    ps = inputs.uniform(100_000, 3)
    pts = gpu_points(ps)
    ws = wg.new_workspace(wg.workspace_size(len(ps)))
    o = wg.default_options(validate=1)
    out = torch.empty(len(ps), dtype=torch.int32, device=DEV)
    cnt = torch.empty(1, dtype=torch.int32, device=DEV)
    wg.upper_hood_into(pts, out, cnt, ws, o)
    assert wg.device_status(ws) == 0
    bad = pts.clone()
    bad[[7000, 7001]] = bad[[7001, 7000]]
    wg.upper_hood_into(bad, out, cnt, ws, o)
    assert wg.device_status(ws) == 3
    bad = pts.clone()
    # 0.3 in float32 is a multiple of 2^-24; one more 2^-25 is off the grid
    # but still below the next grid value, so the order is unchanged.
    bad[9000, 1] = float(np.float32(0.3) + np.float32(2.0 ** -25))
    wg.upper_hood_into(bad, out, cnt, ws, o)
    assert wg.device_status(ws) == 4


def test_timeout_hook(wg):
    ps = inputs.uniform(200_000, 3)
    pts = gpu_points(ps)
    ws = wg.new_workspace(wg.workspace_size(len(ps)))
    wg.debug_set_stall(ws, 2_000_000)  # 2 ms bounded wait that nothing ends
    out = torch.empty(len(ps), dtype=torch.int32, device=DEV)
    cnt = torch.empty(1, dtype=torch.int32, device=DEV)
    wg.upper_hood_into(pts, out, cnt, ws)
    assert wg.device_status(ws) == 5
    wg.debug_set_stall(ws, 0)
    got = wg.upper_hood(pts, workspace=ws).cpu().numpy()
    assert_same(got, oracle.upper_hull(ps.kx, ps.ky), "after timeout")
    assert wg.device_status(ws) == 0


def test_from_host(wg):
    ps = inputs.uniform(1 << 20, 8)
    n = len(ps)
    h_pts = ps.points()
    d_pts = torch.empty((n, 2), dtype=torch.float32, device=DEV)
    d_out = torch.empty(n, dtype=torch.int32, device=DEV)
    d_cnt = torch.empty(1, dtype=torch.int32, device=DEV)
    ws = wg.new_workspace(wg.workspace_size(n))
    h_out = np.empty(n, dtype=np.int32)
    h = wg.upper_hood_from_host(h_pts, d_pts, d_out, d_cnt, ws, h_out)
    assert_same(h_out[:h], oracle.upper_hull(ps.kx, ps.ky), "from host")


def test_autotune_keeps_results(wg):
    ps = inputs.uniform(1 << 22, 12)
    pts = gpu_points(ps)
    best = wg.autotune(pts)
    assert 1 <= best.tile_config <= 4
    got = wg.upper_hood(pts).cpu().numpy()
    assert_same(got, oracle.upper_hull(ps.kx, ps.ky), "after autotune")


# ---------------------------------------------------------------- convex hull
@pytest.mark.parametrize("kind", KINDS)
def test_convex_hull_small_and_tile_edges(wg, kind):
    ws = wg.new_workspace(wg.convex_hull_workspace_size(1 << 20))
    sizes = list(range(0, 120)) + [479, 480, 481, 991, 992, 993, 5000, 100_003, 1 << 20]
    for n in sizes:
        ps = inputs.make(kind, n, 500 + n)
        pts = gpu_points(ps) if n else torch.empty((0, 2), dtype=torch.float32, device=DEV)
        got = wg.convex_hull(pts, workspace=ws).cpu().numpy()
        assert_same(got, oracle.convex_hull(ps.kx, ps.ky), f"hull {kind} n={n}")
    assert wg.device_status(ws) == 0


@pytest.mark.parametrize("name,make", [
    ("2^24 uniform", lambda: inputs.uniform(1 << 24, 2)),
    ("2^24 arc", lambda: inputs.arc(1 << 24, 3)),
    ("closed form", lambda: inputs.closed_form()),
    ("2^26 band", lambda: inputs.band(1 << 26, 4)),
])
def test_convex_hull_configs(wg, name, make):
    ps = make()
    got = wg.convex_hull(gpu_points(ps)).cpu().numpy()
    assert_same(got, oracle.convex_hull(ps.kx, ps.ky), f"hull {name}")


# ---------------------------------------------------------------- shards (the multi-GPU exchange)
@pytest.mark.parametrize("kind", ["uniform", "band", "arc", "duplicates", "columns", "gauss_x"])
@pytest.mark.parametrize("k", [2, 3, 8])
def test_virtual_shards_then_merge(wg, kind, k):
    # The exchange a sharded run would make, on one GPU: k contiguous shards
    # of one set are hulled by separate wg_upper_hood calls (as k ranks
    # would), their corners (coordinates and global indices) are gathered in
    # shard order, and one more call hulls the gathered corners. The hood of
    # a union is the hood of the union of the shards' hoods, and repeats that
    # straddle a shard boundary keep their first occurrence.
    n = 1_000_003
    ps = inputs.make(kind, n, 70 + k)
    pts = gpu_points(ps)
    ws = wg.new_workspace(wg.workspace_size(n))
    gathered = []
    for r in range(k):
        lo, hi = r * n // k, (r + 1) * n // k
        h = wg.upper_hood(pts[lo:hi], workspace=ws)
        gathered.append(h.to(torch.int64) + lo)
    cand = torch.cat(gathered)
    merged = wg.upper_hood(pts[cand].contiguous(), workspace=ws)
    got = cand[merged.to(torch.int64)].cpu().numpy()
    assert_same(got, oracle.upper_hull(ps.kx, ps.ky), f"{k} shards of {kind}")
    assert wg.device_status(ws) == 0


# ---------------------------------------------------------------- huge hoods (multi-level bridge)
def _convex_chain(L):
    # a strictly convex lattice chain: every primitive step (a, b) with
    # a >= 1, |b| <= a and a + |b| <= L, by decreasing slope b / a
    from math import gcd
    steps = [(a, b) for a in range(1, L + 1) for b in range(-a, a + 1) if a + abs(b) <= L and gcd(a, abs(b)) == 1]
    steps.sort(key=lambda v: -v[1] / v[0])
    kx = np.concatenate([[0], np.cumsum([v[0] for v in steps])]).astype(np.int64)
    ky = np.concatenate([[0], np.cumsum([v[1] for v in steps])]).astype(np.int64)
    return kx, ky - ky.min()


@pytest.mark.parametrize("L", [60, 120, 330])
def test_bridge_cta_huge_hoods(wg, L):
    # two convex chains of 10^3..3 10^4 corners, the second shifted right and
    # by a random height, so that the bridge falls anywhere along both; the
    # CTA search (multi-level bracketing) and the warp search must both give
    # the oracle's bridge
    kx, ky = _convex_chain(L)
    m = kx.shape[0]
    assert kx[-1] < inputs.G // 2 and ky.max() < inputs.G // 4
    r = np.random.default_rng(L)
    for trial in range(6):
        a = int(r.integers(m // 4, m))
        b = int(r.integers(m // 4, m))
        dx = int(kx[a - 1]) + int(r.integers(1, 1000))
        dy = int(r.integers(-int(ky.max()) // 2, int(ky.max()) // 2))
        px, py = kx[:a], ky[:a] + inputs.G // 4
        qx, qy = kx[:b] + dx, ky[:b] + inputs.G // 4 + dy
        ref = oracle.bridge(px, py, qx, qy)
        P = torch.from_numpy(inputs.to_float_points(px, py)).to(DEV)
        Q = torch.from_numpy(inputs.to_float_points(qx, qy)).to(DEV)
        assert wg.debug_bridge_cta(P, Q) == ref, (L, trial, a, b)
        assert wg.debug_bridge_cta(P, Q, pred_mode=1) == ref
        if a < 5000:
            assert wg.debug_bridge(P, Q) == ref


def test_bridge_cta_against_oracle_random(wg):
    # the CTA search on the same hood pairs as the warp search tests
    for kind in ("fine", "coarse", "arc", "concave"):
        r = np.random.default_rng({"fine": 2, "coarse": 3, "arc": 13, "concave": 14}[kind] + 100)
        for trial in range(150):
            n = int(r.integers(2, {"arc": 400, "concave": 600}.get(kind, 3000)))
            span = int(r.integers(2, 64)) if kind == "coarse" else inputs.G
            pair = _hood_pair(r, n, span, kind)
            if pair is None:
                continue
            kx, ky, hp, hq = pair
            ref = oracle.bridge(kx[hp], ky[hp], kx[hq], ky[hq])
            P = torch.from_numpy(inputs.to_float_points(kx[hp], ky[hp])).to(DEV)
            Q = torch.from_numpy(inputs.to_float_points(kx[hq], ky[hq])).to(DEV)
            assert wg.debug_bridge_cta(P, Q) == ref, (kind, trial)


# ---------------------------------------------------------------- unsorted input (device sort)
def _shuffled(ps, seed):
    r = np.random.default_rng(seed)
    order = r.permutation(len(ps.kx))
    return ps.kx[order], ps.ky[order]


def _grid_points(kx, ky):
    return torch.from_numpy(np.stack([kx, ky], axis=1).astype(np.float32) * np.float32(2.0 ** -24)).to(DEV)


@pytest.mark.parametrize("kind", ["uniform", "duplicates", "columns", "gauss_x", "band"])
def test_sort_points(wg, kind):
    # The permutation of a stable sort by (x, y) is unique: compared whole
    # with the oracle's.
    for n in (1, 2, 31, 4095, 4096, 4097, 100_003, 1_000_000):
        kx, ky = _shuffled(inputs.make(kind, n, n + 1), n)
        ref = oracle.sort_points(kx, ky)
        sp, perm = wg.sort_points(_grid_points(kx, ky))
        assert np.array_equal(perm.cpu().numpy(), ref), f"{kind} n={n}"
        want = np.stack([kx[ref], ky[ref]], axis=1).astype(np.float32) * np.float32(2.0 ** -24)
        assert np.array_equal(sp.cpu().numpy(), want), f"{kind} n={n} points"


@pytest.mark.parametrize("kind", ["uniform", "arc", "duplicates", "columns", "gauss_x", "band"])
def test_upper_hood_unsorted(wg, kind):
    # corners of shuffled input, as input indices: the oracle on the stably
    # sorted points, mapped back through the sort's permutation (a repeated
    # point counts by its first copy in the input)
    for n in (1, 5, 300, 8192, 8193, 250_001):
        kx, ky = _shuffled(inputs.make(kind, n, n + 2), n + 9)
        order = oracle.sort_points(kx, ky)
        ref = order[oracle.upper_hull(kx[order], ky[order])].astype(np.int32)
        got = wg.upper_hood_unsorted(_grid_points(kx, ky)).cpu().numpy()
        assert_same(got, ref, f"{kind} n={n}")


def test_sort_points_large(wg):
    kx, ky = _shuffled(inputs.uniform(1 << 24, 2), 3)
    ref = oracle.sort_points(kx, ky)
    _, perm = wg.sort_points(_grid_points(kx, ky))
    assert np.array_equal(perm.cpu().numpy(), ref)
