"""Benchmark of the upper-hood path on GB300 (prints one JSON line).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload uniform26|uniform24|arc24|band26|gauss28|uniform16|closed4096|batched]

A step is one pass of the whole path over one input: one call of
wg_upper_hood on a device-resident set (one fused kernel launch). The default
workload is one set of 2^26 points uniform on the 2^-24 grid (537 MB, larger
than the 129 MB L2, so no flush is needed between steps).

value      = points processed by all ranks / (max over ranks of the timed
             region), Gpoints/s, timed with CUDA events on the launching
             stream around K steps after W warm-up steps.
e2e        = the same metric through wg_upper_hood_from_host: pinned host
             points copied in, corners and count copied out, every step.
roofline   = algorithmic bytes (8n in + 4h + 4 out) per launch / median
             launch time (>= 20 launches, CUDA events on both sides of each,
             in a loop after the timed one), against the measured HBM copy
             bandwidth.
cpu_baseline = the CPU oracle's monotone chain run strip-parallel on every
             host core, on the same input (the single-thread time is
             reported beside it).

Under torchrun (N > 1) every rank hulls its own set of the same size (weak
scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "upper-hull Gpoints/s and % HBM roofline; batched sets/s vs plain per-set"
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "uniform26": ("uniform", 1 << 26, 7, "uniform n=2^26 single set"),
    "uniform24": ("uniform", 1 << 24, 2, "uniform n=2^24 single set"),
    "arc24": ("arc", 1 << 24, 3, "arc y=1-4(x-1/2)^2 n=2^24 single set"),
    "band26": ("band", 1 << 26, 4, "parabola band 2^-20 wide n=2^26 single set"),
    "gauss28": ("gauss_x", 1 << 28, 6, "gaussian-x n=2^28 single set"),
    "uniform16": ("uniform", 1 << 16, 1, "uniform n=2^16 single set"),
    "closed4096": ("closed_form", 4096, 0, "closed form x=i/4096, y=i(4095-i)/2^24"),
}


def _code_only(text: str) -> str:
    """C++ source without comments and with whitespace collapsed."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


# The sources that define the fused kernel (device code and its instantiations).
KERNEL_SOURCES = ("wg_device.cuh", "wg_fused.cuh", "wg_internal.h", "wg_fused.cu", "wg_fused_cfg1.cu",
                  "wg_fused_cfg2.cu", "wg_fused_cfg3.cu", "wg_fused_cfg4.cu", "wg_small.cu")
SMALL_MAX_N = 8192  # the library's default path up to this size is the one-CTA small kernel


def kernel_source_hash() -> str:
    """Hash of the fused kernel's sources (code only: comments and layout
    ignored), which ties a committed ncu summary to the kernel it measured."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1203_5004_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in KERNEL_SOURCES:
            with open(os.path.join(csrc, name), encoding="utf-8") as f:
                h.update(name.encode() + b"\0" + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic_per_point(workload: str):
    """dram bytes per input point from a committed ncu summary of a smaller
    case of the same workload, if it matches this kernel."""
    path = os.path.join(ROOT, "profiles", f"fused_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_point:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


def profiled_traffic(workload: str, kernel: str = "fused"):
    """dram bytes per launch from the committed ncu summary, if it matches this source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_source_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        ident = str(self.dev)
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(self.dev).uuid)
            ident = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", ident], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank float over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank r's set under weak scaling (rank 0 uses the workload's own)."""
    return seed + 1000 * rank if rank else seed


def make_input(kind: str, n: int, seed: int):
    from paper_1203_5004_gb300 import inputs
    return inputs.make(kind, n, seed)


def time_oracle(ps, budget_s: float = 12.0, max_reps: int = 20):
    """The CPU oracle as it stands, one core, repeated on the full input."""
    import oracle
    oracle.upper_hull(ps.kx[:1000], ps.ky[:1000])  # build + load outside the timing
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.upper_hull(ps.kx, ps.ky)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= max_reps:
            break
    return len(ps) * reps / el / 1e9, reps, el


def time_oracle_strips(ps, budget_s: float = 8.0, max_reps: int = 40):
    """The oracle's chain run strip-parallel on every host core (one strip
    per core, then one chain over the strip hoods), repeated on the full
    input. Returns (Gpoints/s, reps, seconds, cores)."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.upper_hull_strips(ps.kx[:1000], ps.ky[:1000], cores)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.upper_hull_strips(ps.kx, ps.ky, cores)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= max_reps:
            break
    return len(ps) * reps / el / 1e9, reps, el, cores


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle timed as the step, on this workload."""
    if rank != 0:
        return
    if args.workload == "batched":
        from paper_1203_5004_gb300 import inputs
        import oracle
        S = args.sets
        ps, offs, _ = inputs.batched(S, seed=5)
        oracle.upper_hull(ps.kx[:1000], ps.ky[:1000])
        t0 = time.perf_counter()
        oracle.upper_hull_batched(ps.kx, ps.ky, offs)
        el = time.perf_counter() - t0
        value = S / el
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "sets/s", "n_gpus": world,
            "steps": 1, "warmup": 0, "ms_per_step": el * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"batched {S} sets, sizes log-uniform in [3, 65536], mixed kinds", "sets": S,
                       "points": int(offs[-1]), "seed": 5},
            "cpu_baseline": {"value": value, "unit": "sets/s", "cores": 1, "kind": "oracle",
                             "sample": f"all {S} sets once, single-thread monotone chain"},
            "e2e": {"value": value, "unit": "sets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    if args.workload == "sort26":
        _, kxy = sort_input(0)
        value, reps, el, _ = time_argsort(kxy, budget_s=30.0, max_reps=max(1, min(args.steps, 5)))
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world,
            "steps": reps, "warmup": 0, "ms_per_step": el / reps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "device sort of 2^26 uniform grid points in random order (48-bit keys)",
                       "n": SORT_N, "seed": SORT_SEED},
            "cpu_baseline": {"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle (stable sort of the 48-bit keys)",
                             "sample": f"full input, {reps} runs"},
            "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    if args.workload in ("hull26", "bridge_cta"):
        import oracle
        reps = max(1, min(args.steps, 5))
        if args.workload == "hull26":
            kind, n, seed, desc = WORKLOADS["uniform26"]
            ps = make_input(kind, n, seed)
            t0 = time.perf_counter()
            for _ in range(reps):
                oracle.convex_hull(ps.kx, ps.ky)
            el = time.perf_counter() - t0
            value, unit, wl = n * reps / el / 1e9, "Gpoints/s", "convex hull of the " + desc
        else:
            from paper_1203_5004_gb300 import inputs
            kx, ky = convex_chain(330)
            px, py = kx, ky + inputs.G // 4
            qx, qy = kx + int(kx[-1]) + 500, ky + inputs.G // 4 + int(ky.max()) // 3
            t0 = time.perf_counter()
            for _ in range(reps):
                oracle.bridge(px, py, qx, qy)
            el = time.perf_counter() - t0
            value, unit, wl = reps / el, "bridges/s", f"bridge of two convex chains of {kx.shape[0]} corners each"
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": reps,
            "warmup": 0, "ms_per_step": el / reps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": {"workload": wl},
            "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "sample": f"{reps} runs"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line), flush=True)
        return
    kind, n, seed, desc = WORKLOADS[args.workload]
    ps = make_input(kind, n, seed)
    import oracle
    oracle.upper_hull(ps.kx[:1000], ps.ky[:1000])
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.upper_hull(ps.kx, ps.ky)
    steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle.upper_hull(ps.kx, ps.ky)
    el = time.perf_counter() - t0
    value = n * steps / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpoints/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": el / steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": desc, "n": n, "seed": seed},
        "cpu_baseline": {"value": value, "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
                         "sample": f"full input, {steps} runs of the single-thread monotone chain"},
        "e2e": {"value": value, "unit": "Gpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


SORT_N, SORT_SEED = 1 << 26, 8


def sort_input(rank: int):
    """2^26 uniform grid points in a seeded random order (the sort workload):
    the float32 points and their integer coordinates."""
    from paper_1203_5004_gb300 import inputs
    ps = inputs.uniform(SORT_N, rank_seed(SORT_SEED, rank))
    order = np.random.default_rng(rank_seed(SORT_SEED + 1, rank)).permutation(SORT_N)
    kx, ky = ps.kx[order], ps.ky[order]
    pts = np.stack([kx, ky], axis=1).astype(np.float32) * np.float32(2.0 ** -24)
    return pts, (kx, ky)


def time_argsort(kxy, budget_s=20.0, max_reps=5):
    """The sort oracle as it stands (a stable sort of the 48-bit keys, one core)."""
    import oracle
    kx, ky = kxy
    reps, t0 = 0, time.perf_counter()
    ref = None
    while reps < max_reps and (reps == 0 or time.perf_counter() - t0 < budget_s):
        ref = oracle.sort_points(kx, ky)
        reps += 1
    el = time.perf_counter() - t0
    return kx.size * reps / el / 1e9, reps, el, ref


def run_sort(args, world, rank, local):
    """The device sort of unsorted points (the step before the path)."""
    import ctypes
    import torch
    from paper_1203_5004_gb300 import _lib, wagener
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    n = SORT_N
    h_pts, kxy = sort_input(rank)
    pts = torch.from_numpy(h_pts).to(dev)
    ws = wagener.new_workspace(wagener.sort_points_workspace_size(n), dev)
    out = torch.empty((n, 2), dtype=torch.float32, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib = _lib.load()

    def step():
        _lib.check(lib.wg_sort_points(pts.data_ptr(), n, out.data_ptr(), perm.data_ptr(), ws.data_ptr(), ws.numel(),
                                      stream.cuda_stream), "wg_sort_points")
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    K = max(1, min(args.steps, 50))
    if args.profile:
        for _ in range(K):
            step()
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"profile_run": True, "workload": "sort uniform 2^26", "n": n, "steps": K}))
        return
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(K):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    total_ms = max_over_ranks(t0.elapsed_time(t1), pg, dev)
    value = n * world * K / (total_ms * 1e-3) / 1e9
    nl = 20
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nl)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nl)]
    for i in range(nl):
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    call_ms = float(np.median([a.elapsed_time(b) for a, b in zip(starts, ends)]))
    # end to end: points from pinned host memory, the sort, the permutation back
    hp = torch.from_numpy(h_pts).pin_memory()
    hperm = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_steps = 5
    torch.cuda.synchronize(dev)
    te = time.perf_counter()
    for _ in range(e2e_steps):
        pts.copy_(hp, non_blocking=True)
        step()
        hperm.copy_(perm, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_value = n * world * e2e_steps / (time.perf_counter() - te) / 1e9
    if pg:
        pg.barrier()
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    cpu, reps, el, ref = time_argsort(kxy)
    same = bool(np.array_equal(hperm.numpy(), ref))
    peak, peak_kind = measured_peak()
    alg_bytes = 8 * n + 12 * n  # points read once, sorted points and permutation written once
    achieved = alg_bytes / (call_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "device sort of 2^26 uniform grid points in random order (48-bit keys)", "n": n,
                   "seed": SORT_SEED, "passes": 6, "same_permutation_as_oracle": same,
                   "l2": "input 8n bytes > 129 MB L2 (no flush)", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_source": peak_kind, "kernel": "wg_sort_points (all launches of one call)",
                     "alg_bytes_per_launch": alg_bytes, "launch_ms_median": call_ms, "launches_timed": nl},
        "e2e": {"value": e2e_value, "unit": "Gkeys/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 4 * n},
        "gpu_launches": K * 32,
        "clocks": clocks,
        "cpu_baseline": {"value": cpu, "unit": "Gkeys/s", "cores": 1, "kind": "oracle (stable sort of the 48-bit keys)",
                         "sample": f"full input, {reps} runs, {el:.1f} s"},
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def run_hull(args, world, rank, local):
    """The full convex hull (the title problem) of the 2^26 uniform set."""
    import torch
    from paper_1203_5004_gb300 import _lib, wagener
    import oracle
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    kind, n, seed, desc = WORKLOADS["uniform26"]
    ps = make_input(kind, n, rank_seed(seed, rank))
    h_pts = ps.points()
    pts = torch.from_numpy(h_pts).to(dev)
    ws = wagener.new_workspace(wagener.convex_hull_workspace_size(n), dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib = _lib.load()

    def step():
        _lib.check(lib.wg_convex_hull(pts.data_ptr(), n, out.data_ptr(), cnt.data_ptr(), ws.data_ptr(), ws.numel(),
                                      None, stream.cuda_stream), "wg_convex_hull")
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    h = int(cnt.item())
    K = max(1, min(args.steps, 500))
    if args.profile:
        for _ in range(K):
            step()
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"profile_run": True, "workload": "convex hull " + desc, "n": n, "steps": K}))
        return
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(K):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    total_ms = max_over_ranks(t0.elapsed_time(t1), pg, dev)
    value = n * world * K / (total_ms * 1e-3) / 1e9
    nl = 20
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nl)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nl)]
    for i in range(nl):
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    call_ms = float(np.median([a.elapsed_time(b) for a, b in zip(starts, ends)]))
    hp = torch.from_numpy(h_pts).pin_memory()
    hout = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_steps = 5
    torch.cuda.synchronize(dev)
    te = time.perf_counter()
    for _ in range(e2e_steps):
        pts.copy_(hp, non_blocking=True)
        step()
        hh = int(cnt.item())
        hout[:hh].copy_(out[:hh])
    torch.cuda.synchronize(dev)
    e2e_value = n * world * e2e_steps / (time.perf_counter() - te) / 1e9
    if pg:
        pg.barrier()
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    reps, tc = 0, time.perf_counter()
    ref = None
    while reps < 5 and (reps == 0 or time.perf_counter() - tc < 20.0):
        ref = oracle.convex_hull(ps.kx, ps.ky)
        reps += 1
    el = time.perf_counter() - tc
    same = bool(np.array_equal(hout[:h].numpy(), ref))
    peak, peak_kind = measured_peak()
    # two upper-hood passes over the points, the turned copy written once, the corners
    alg_bytes = 8 * n + 8 * n + 8 * n + 4 * h + 4
    achieved = alg_bytes / (call_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "Gpoints/s", "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "convex hull of the " + desc, "n": n, "seed": seed, "hull_corners": h,
                   "same_corners_as_oracle": same, "l2": "input 8n bytes > 129 MB L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_source": peak_kind, "kernel": "wg_convex_hull (all launches of one call)",
                     "alg_bytes_per_launch": alg_bytes, "launch_ms_median": call_ms, "launches_timed": nl},
        "e2e": {"value": e2e_value, "unit": "Gpoints/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 4 + 4 * h},
        "gpu_launches": K * 5,
        "clocks": clocks,
        "cpu_baseline": {"value": n * reps / el / 1e9, "unit": "Gpoints/s", "cores": 1,
                         "kind": "oracle (upper and lower monotone chains)", "sample": f"full input, {reps} runs"},
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def convex_chain(L: int):
    """A strictly convex lattice chain: every primitive step (a, b) with
    a >= 1, |b| <= a and a + |b| <= L, by decreasing slope (a hood of many
    thousands of corners for the bridge searches)."""
    from math import gcd
    steps = [(a, b) for a in range(1, L + 1) for b in range(-a, a + 1) if a + abs(b) <= L and gcd(a, abs(b)) == 1]
    steps.sort(key=lambda v: -v[1] / v[0])
    kx = np.concatenate([[0], np.cumsum([v[0] for v in steps])]).astype(np.int64)
    ky = np.concatenate([[0], np.cumsum([v[1] for v in steps])]).astype(np.int64)
    return kx, ky - ky.min()


def run_bridge(args, world, rank, local):
    """The bridge of two huge hoods (paper Section 2, mam 1-5): the CTA's
    multi-level bracketing search against the one-warp search."""
    import torch
    from paper_1203_5004_gb300 import inputs, wagener
    import oracle
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kx, ky = convex_chain(330)
    m = int(kx.shape[0])
    dx = int(kx[-1]) + 500
    px, py = kx, ky + inputs.G // 4
    qx, qy = kx + dx, ky + inputs.G // 4 + int(ky.max()) // 3
    ref = oracle.bridge(px, py, qx, qy)
    P = torch.from_numpy(inputs.to_float_points(px, py)).to(dev)
    Q = torch.from_numpy(inputs.to_float_points(qx, qy)).to(dev)
    stream = torch.cuda.current_stream(dev)
    from paper_1203_5004_gb300 import _lib
    lib = _lib.load()
    pq = torch.empty(2, dtype=torch.int32, device=dev)
    res = {}
    K = max(1, min(args.steps, 200))
    for name, fn, raw in (("cta", wagener.debug_bridge_cta, lib.wg_debug_bridge_cta),
                          ("warp", wagener.debug_bridge, lib.wg_debug_bridge)):
        res[name + "_same"] = bool(tuple(fn(P, Q)) == tuple(ref))

        def call():
            _lib.check(raw(P.data_ptr(), m, Q.data_ptr(), m, pq.data_ptr(), 0, stream.cuda_stream), name)
        for _ in range(3):
            call()
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            call()
        b.record(stream)
        torch.cuda.synchronize(dev)
        res[name + "_us"] = a.elapsed_time(b) / K * 1e3
    if rank != 0:
        return
    tc = time.perf_counter()
    for _ in range(20):
        oracle.bridge(px, py, qx, qy)
    cpu_us = (time.perf_counter() - tc) / 20 * 1e6
    line = {
        "metric": METRIC, "value": 1e6 / res["cta_us"], "unit": "bridges/s", "n_gpus": 1, "steps": K,
        "warmup": 1, "ms_per_step": res["cta_us"] / 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"bridge of two convex chains of {m} corners each (one launch per bridge, "
                               "back to back on the device)",
                   "corners_per_hood": m, "same_bridge_as_oracle": res["cta_same"] and res["warp_same"]},
        "roofline": {"bound": "latency", "achieved": None, "peak": None, "unit": None, "frac": None,
                     "traffic": None, "kernel": "bridge_cta (one CTA)"},
        "compare": {"warp_search_us": res["warp_us"], "cta_search_us": res["cta_us"]},
        "e2e": {"value": None, "unit": "bridges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8},
        "gpu_launches": K,
        "cpu_baseline": {"value": 1e6 / cpu_us, "unit": "bridges/s", "cores": 1, "kind": "oracle (monotone chain "
                         "over both hoods)", "sample": "20 runs"},
    }
    print(json.dumps(line), flush=True)


DEFAULT_COMPARE = {
    "band26": ("counters", "fp64_only"),
    "gauss28": ("plain",),
}


def time_steps(fn, steps, stream, dev):
    """Average ms per call of fn over `steps` calls, CUDA events on `stream`."""
    import torch
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / steps


def run_batched(args, world, rank, local):
    """Many sets in one launch vs one wg_upper_hood call per set."""
    import ctypes

    import torch
    from paper_1203_5004_gb300 import _lib, inputs, wagener

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    S = args.sets
    ps, offs, _ = inputs.batched(S, seed=rank_seed(5, rank))
    total = int(offs[-1])
    pts = torch.from_numpy(ps.points()).to(dev)
    offs_d = torch.from_numpy(offs).to(dev)
    out = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    counts = torch.empty(max(S, 1), dtype=torch.int32, device=dev)
    ws = wagener.new_workspace(wagener.batched_workspace_size(offs), dev)
    stream = torch.cuda.current_stream(dev)
    if args.tile_config:
        bopts = wagener.default_options(tile_config=args.tile_config, batch_seg_tiles=args.batch_seg_tiles)
    elif args.no_autotune:
        bopts = None
    else:
        bopts = wagener.autotune_batched(pts, offs_d, ws)
    direct = lambda: wagener.upper_hood_batched_into(pts, offs_d, out, counts, ws, bopts)
    for _ in range(max(3, args.warmup)):
        direct()
    torch.cuda.synchronize(dev)
    if args.profile:
        for _ in range(args.steps):
            direct()
        torch.cuda.synchronize(dev)
        return
    ref_counts = counts.clone()
    # One step (two planning kernels + the persistent fused kernel) captured in a CUDA
    # graph; the workspace's counters reset themselves, so replays are exact.
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        direct()
    torch.cuda.synchronize(dev)
    step = graph.replay
    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    graph_same = bool(torch.equal(counts, ref_counts))
    K = args.steps
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    ms = time_steps(step, K, stream, dev)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, pg, dev)
    direct_ms = time_steps(direct, K, stream, dev)
    value = S * world / (ms * 1e-3)
    hsum = int(counts.sum().item())

    # End to end: every step copies its inputs from pinned host memory,
    # hulls them and reads the per-set counts back. Two device buffers and a
    # copy stream let step k+1's copy run under step k's hull, as a serving
    # loop would; each step still moves all of its bytes.
    pts_h = pts.cpu().pin_memory()
    offs_h = offs_d.cpu().pin_memory()
    counts_h = [torch.empty_like(counts, device="cpu").pin_memory() for _ in range(2)]
    pts_b = [pts, torch.empty_like(pts)]
    offs_b = [offs_d, torch.empty_like(offs_d)]
    counts_b = [counts, torch.empty_like(counts)]
    copy_stream = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    for d_ in done:
        d_.record(stream)

    def e2e_run(k_steps):
        copy_stream.wait_stream(stream)  # no copy starts before the timed region
        for k in range(k_steps):
            b = k & 1
            copy_stream.wait_event(done[b])
            with torch.cuda.stream(copy_stream):
                pts_b[b].copy_(pts_h, non_blocking=True)
                offs_b[b].copy_(offs_h, non_blocking=True)
                copied[b].record(copy_stream)
            stream.wait_event(copied[b])
            wagener.upper_hood_batched_into(pts_b[b], offs_b[b], out, counts_b[b], ws, bopts)
            counts_h[b].copy_(counts_b[b], non_blocking=True)
            done[b].record(stream)
    e2e_run(2)
    torch.cuda.synchronize(dev)
    e2e_k = max(2, min(K, 6))
    e2e_ms = max_over_ranks(time_steps(lambda: e2e_run(e2e_k), 1, stream, dev) / e2e_k, pg, dev)
    e2e_same = all(bool(torch.equal(c_, ref_counts.cpu())) for c_ in counts_h)

    # The plain per-set form: one wg_upper_hood call per set, same GPU.
    lib = _lib.load()
    wsz = lib.wg_upper_hood_workspace_size(0)
    pws = torch.zeros(wsz, dtype=torch.uint8, device=dev)
    pout = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    pcnt = torch.empty(max(S, 1), dtype=torch.int32, device=dev)
    base_p, base_o, base_c = pts.data_ptr(), pout.data_ptr(), pcnt.data_ptr()
    sc = stream.cuda_stream
    fn = lib.wg_upper_hood

    def plain_sets():
        for s_ in range(S):
            a_, b_ = int(offs[s_]), int(offs[s_ + 1])
            fn(base_p + 8 * a_, b_ - a_, base_o + 4 * a_, base_c + 4 * s_, pws.data_ptr(), wsz, sc)
    plain_sets()
    plain_ms = time_steps(plain_sets, 1, stream, dev)
    same = bool(torch.equal(pcnt[:S], counts[:S]))
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.upper_hull_batched_threads(ps.kx, ps.ky, offs, cores)
    cpu_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.upper_hull_batched(ps.kx, ps.ky, offs)
    cpu1_s = time.perf_counter() - t0
    peak, peak_kind = measured_peak()
    alg = 8 * total + 4 * hsum + 8 * (S + 1) + 4 * S
    per_point = profiled_traffic_per_point("batched")
    traffic = per_point * total if per_point is not None else None
    line = {
        "metric": METRIC, "value": value, "unit": "sets/s", "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched {S} sets, sizes log-uniform in [3, 65536], mixed kinds",
                   "sets": S, "points": total, "corners": hsum, "seed": 5,
                   "tile_config": int(bopts.tile_config) if bopts else 0,
                   "batch_seg_tiles": int(bopts.batch_seg_tiles) if bopts else 0,
                   "gpoints_per_s": total / (ms * 1e-3) / 1e9, "cuda_graph": True,
                   "l2": "input > 129 MB L2 (no flush)", "parallelism": f"replicas x{world}"},
        "compare": {"plain_per_set_ms_per_step": plain_ms, "plain_per_set_sets_per_s": S / (plain_ms * 1e-3),
                    "batched_speedup": plain_ms / ms, "plain_counts_equal": same,
                    "direct_launch_ms_per_step": direct_ms, "graph_counts_equal": graph_same},
        "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg / (ms * 1e-3) / 1e9 / peak, "traffic": traffic, "peak_source": peak_kind,
                     "kernel": "fused_kernel (batched)", "alg_bytes_per_launch": alg},
        "e2e": {"value": S * world / (e2e_ms * 1e-3), "unit": "sets/s",
                "h2d_bytes_per_step": 8 * total + 8 * (S + 1), "d2h_bytes_per_step": 4 * S,
                "counts_equal": e2e_same},
        "gpu_launches": 3 * K,
        "clocks": clocks,
        "cpu_baseline": {"value": S / cpu_s, "unit": "sets/s", "cores": cores,
                         "kind": "oracle, monotone chain per set, sets spread over the host cores",
                         "sample": f"all {S} sets once on {cores} threads, {cpu_s:.2f} s",
                         "single_thread": {"value": S / cpu1_s, "unit": "sets/s", "cores": 1,
                                           "sample": f"all {S} sets once, {cpu1_s:.1f} s"}},
    }
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def run_ours(args, world, rank, local):
    import torch
    from paper_1203_5004_gb300 import wagener

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    kind, n, seed, desc = WORKLOADS[args.workload]
    ps = make_input(kind, n, rank_seed(seed, rank))
    pts = torch.from_numpy(ps.points()).to(dev)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(1, dtype=torch.int32, device=dev)
    ws = wagener.new_workspace(wagener.workspace_size(n), dev)
    stream = torch.cuda.current_stream(dev)

    if args.tile_config:
        opts = wagener.default_options(tile_config=args.tile_config, schedule=args.schedule,
                                       segments_per_cta=args.segments_per_cta)
    elif args.no_autotune:
        opts = wagener.default_options()
    else:
        opts = wagener.autotune(pts, workspace=ws)
    for _ in range(max(3, args.warmup)):
        wagener.upper_hood_into(pts, out, cnt, ws, opts)
    torch.cuda.synchronize(dev)
    h = int(cnt.item())
    if wagener.device_status(ws) != 0:
        raise RuntimeError("device reported an error during warm-up")

    K = args.steps
    if args.profile:
        # Launch list / counter capture: the timed steps only, nothing else.
        for _ in range(K):
            wagener.upper_hood_into(pts, out, cnt, ws, opts)
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"profile_run": True, "workload": desc, "n": n, "steps": K, "hull_corners": h}))
        if pg:
            pg.destroy_process_group()
        return
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    # The timed region: K calls back to back, events only at its ends.
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(K):
        wagener.upper_hood_into(pts, out, cnt, ws, opts)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    total_ms = t0.elapsed_time(t1)
    # Per-launch durations for the roofline, in a separate loop (an event
    # on each side of every launch): the median of at least 20.
    nl = max(20, min(K, 200))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(nl)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(nl)]
    for i in range(nl):
        starts[i].record(stream)
        wagener.upper_hood_into(pts, out, cnt, ws, opts)
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    launch_ms = float(np.median([s.elapsed_time(e) for s, e in zip(starts, ends)]))
    if wagener.device_status(ws) != 0:
        raise RuntimeError("device reported an error in the timed region")
    total_ms = max_over_ranks(total_ms, pg, dev)
    value = n * world * K / (total_ms * 1e-3) / 1e9

    # End to end through the public host-buffer entry point.
    h_pts = torch.from_numpy(ps.points()).pin_memory().numpy()
    h_out = torch.empty(max(n, 1), dtype=torch.int32).pin_memory().numpy()
    e2e_steps = max(1, min(K, 10))
    for _ in range(2):
        wagener.upper_hood_from_host(h_pts, pts, out, cnt, ws, h_out, opts)
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    te = time.perf_counter()
    for _ in range(e2e_steps):
        hh = wagener.upper_hood_from_host(h_pts, pts, out, cnt, ws, h_out, opts)
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - te
    e2e_s = max_over_ranks(e2e_s, pg, dev)
    e2e_value = n * world * e2e_steps / e2e_s / 1e9

    # Other forms of the same step, untimed in `value` (reported in `compare`).
    compare = {}
    wants = set(args.compare.split(",")) if args.compare else set(DEFAULT_COMPARE.get(args.workload, ()))
    if "counters" in wants:
        co = wagener.default_options(tile_config=int(opts.tile_config), segments_per_cta=int(opts.segments_per_cta),
                                     count_predicates=1)
        wagener.read_counters(ws)
        wagener.upper_hood_into(pts, out, cnt, ws, co)
        tests, fb = wagener.read_counters(ws)
        compare["orient_tests"] = tests
        compare["fp64_fallbacks"] = fb
        compare["filter_failure_rate"] = fb / tests if tests else 0.0
    if "fp64_only" in wants:
        fo = wagener.default_options(tile_config=int(opts.tile_config), segments_per_cta=int(opts.segments_per_cta),
                                     pred_mode=1)
        ref = out[:h].clone()
        ms = time_steps(lambda: wagener.upper_hood_into(pts, out, cnt, ws, fo), min(K, 50), stream, dev)
        compare["fp64_only_ms_per_step"] = ms
        compare["fp64_only_gpoints_per_s"] = n / (ms * 1e-3) / 1e9
        compare["fp64_only_same_output"] = bool(int(cnt.item()) == h and torch.equal(out[:h], ref))
    if "plain" in wants:
        pws = wagener.new_workspace(wagener.plain_workspace_size(n), dev)
        pout = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        pcnt = torch.empty(1, dtype=torch.int32, device=dev)

        def plain_step():
            from paper_1203_5004_gb300 import _lib
            import ctypes
            _lib.check(_lib.load().wg_upper_hood_plain(pts.data_ptr(), n, pout.data_ptr(), pcnt.data_ptr(),
                                                       pws.data_ptr(), pws.numel(), None, stream.cuda_stream),
                       "wg_upper_hood_plain")
        plain_step()
        ms = time_steps(plain_step, min(K, 10), stream, dev)
        compare["plain_ms_per_step"] = ms
        compare["plain_gpoints_per_s"] = n / (ms * 1e-3) / 1e9
        compare["plain_launches_per_step"] = max(1, (n - 1).bit_length())
        compare["plain_same_output"] = bool(int(pcnt.item()) == h and torch.equal(pout[:h], out[:h]))
        del pws

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    peak, peak_kind = measured_peak()
    alg_bytes = 8 * n + 4 * h + 4
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    small = int(opts.schedule) == 4 or (int(opts.schedule) == 0 and n <= SMALL_MAX_N)
    kernel = "small_kernel" if small else "fused_kernel"
    traffic = profiled_traffic(args.workload, "small" if small else "fused")
    cpu_gpts, reps, el, cores = time_oracle_strips(ps)
    cpu1_gpts, reps1, el1 = time_oracle(ps, budget_s=6.0, max_reps=10)
    line = {
        "metric": METRIC, "value": value, "unit": "Gpoints/s", "n_gpus": world, "steps": K,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "n": n, "seed": seed, "hull_corners": h,
                   "tile_config": int(opts.tile_config), "segments_per_cta": int(opts.segments_per_cta),
                   "schedule": {1: "balanced", 2: "guided", 3: "one CTA", 4: "small (one CTA, no tiles)"}.get(
                       int(opts.schedule), "library"),
                   "l2": "input 8n bytes > 129 MB L2 (no flush)" if 8 * n > 129e6 else "input fits L2 (no flush)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                     "kernel": kernel, "alg_bytes_per_launch": alg_bytes,
                     "launch_ms_median": launch_ms, "launches_timed": nl},
        "e2e": {"value": e2e_value, "unit": "Gpoints/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 4 + 4 * hh},
        "gpu_launches": K,
        "clocks": clocks,
        "cpu_baseline": {"value": cpu_gpts, "unit": "Gpoints/s", "cores": cores,
                         "kind": "oracle, strip-parallel monotone chain",
                         "sample": f"full input, {reps} runs on {cores} threads, {el:.1f} s",
                         "single_thread": {"value": cpu1_gpts, "unit": "Gpoints/s", "cores": 1,
                                           "sample": f"full input, {reps1} runs, {el1:.1f} s"}},
    }
    if compare:
        line["compare"] = compare
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uniform26",
                    choices=sorted(WORKLOADS) + ["batched", "sort26", "hull26", "bridge_cta"])
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile-config", type=int, default=0, help="fixed tile configuration (0: autotune)")
    ap.add_argument("--profile", action="store_true",
                    help="only warm-up and the K steps (for ncu); prints no bench line")
    ap.add_argument("--compare", default="",
                    help="comma list of extra forms to time: counters, fp64_only, plain")
    ap.add_argument("--sets", type=int, default=100000, help="sets of the batched workload")
    ap.add_argument("--schedule", type=int, default=0,
                    help="single set, with --tile-config: 1 balanced, 2 guided, 3 one CTA, 4 small (0: library choice)")
    ap.add_argument("--segments-per-cta", type=int, default=0,
                    help="single set, with --tile-config: segments per resident warp (0: library choice)")
    ap.add_argument("--batch-seg-tiles", type=int, default=0,
                    help="batched, with --tile-config: tiles per segment of a large set (0: library choice)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "sort26":
        run_sort(args, world, rank, local)
        return
    if args.workload == "hull26":
        run_hull(args, world, rank, local)
        return
    if args.workload == "bridge_cta":
        run_bridge(args, world, rank, local)
        return
    if args.workload == "batched":
        run_batched(args, world, rank, local)
        return
    run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
