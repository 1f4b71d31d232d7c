"""Benchmark: visibility-taps/s and % of the FP32 FMA roofline, coarsened vs plain Romein gridding.

One step is one pass of the whole hot path over one synthetic batch, the
quad-pol workload: G=2048, S=7, O=8, P=4, 8,257,536 baseline-ordered
visibilities. The step zeroes the grid, grids the batch (indices, staging,
sliding-window coarsened accumulation, flushes) and degrids the result (the
adjoint). value = (taps gridded + taps degridded) / s over the timed steps.
Inputs are resident in HBM when the timed region starts. The e2e figure times
the same step through the C ABI from pinned host buffers, with the copies
inside the timed region.

The plain (uncoarsened, B=1) Romein kernel with the paper's schedule (Sec. 4:
1024 visibilities per work-group, flushes straight to global memory) is
timed in the same run on the same inputs.

Usage:
  python bench.py [--gpus N] [--steps K] [--warmup W]   (torchrun for N > 1)
  python bench.py --impl reference ...  times the FP64 CPU oracle on a sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1605_07023_gb300 import synth  # noqa: E402

METRIC = "visibility-taps/s and % FP32 FMA peak, coarsened vs plain Romein, 1 GB300"
UNIT = "vis-taps/s"
WORKLOAD = "quad-pol gridding+degridding: G=2048 S=7 O=8 P=4, 64 antennas (8 km disk), 2016 bl x 1024 t x 4 ch = 8,257,536 vis"
FMA_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="auto", help="grid plan: auto | chunked:Bu,Bv[:vis_per_chunk[:threads]] | patch:Bu,Bv[:vis_per_chunk[:threads]]")
    ap.add_argument("--degrid-config", default="auto", help="degrid plan: auto | chunked:Bu,Bv[:L[:T]] | tile:Bu,Bv:0:T")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--vis", type=int, default=0, help="use only the first N visibilities (profiling runs)")
    ap.add_argument("--skip-plain", action="store_true", help="do not time the plain Romein kernel (profiling runs)")
    ap.add_argument("--no-compression", action="store_true", help="skip the compression measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the coarsening sweep and the single-pol comparison")
    ap.add_argument("--no-extra", action="store_true", help="skip the batching, differentiation and small workloads")
    return ap.parse_args()


def dist_init(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    import torch
    from paper_1605_07023_gb300 import sharding
    return sharding.reduce_max(x, "cuda" if torch.cuda.is_available() else "cpu") if world > 1 else x


def sum_over_ranks(x: float, world: int) -> float:
    import torch
    from paper_1605_07023_gb300 import sharding
    return sharding.reduce_sum(x, "cuda" if torch.cuda.is_available() else "cpu") if world > 1 else x


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def fma_peak_tflops(sm_count: int, max_mhz: float) -> float:
    """FP32 FMA roofline: SMs x 128 FMA lanes x 2 flop x max SM clock."""
    return sm_count * FMA_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12


FLOPS_PER_GPA = 4.0        # real Kaiser-Bessel taps: two FFMA (re, im) per grid-point addition
PAPER_FLOPS_PER_GPA = 8.0  # the paper's count for one grid-point addition (Sec. 5)


def fma_fraction(gpa_per_s: float, peak_tflops: float, flops_per_gpa: float = FLOPS_PER_GPA) -> float:
    """Fraction of an FP32 peak reached at a rate of grid-point additions (one polarization's
    multiply-accumulate into one cell) per second."""
    return gpa_per_s * flops_per_gpa / (peak_tflops * 1e12)


def cpu_oracle_rate(w, n_sample: int, table64):
    """Time the FP64 oracle (single thread, as it stands) on the first n_sample visibilities: grid + degrid."""
    import oracle
    oracle.build()
    sub = synth.scaled_down(w, n_sample)
    t0 = time.perf_counter()
    g, sk = oracle.grid(w.G, w.S, w.oversample, sub.uv, sub.vis, sub.weights, table64)
    oracle.degrid(w.G, w.S, w.oversample, sub.uv, g, table64)
    dt = time.perf_counter() - t0
    n_valid = n_sample - sk
    return 2 * n_valid * w.S * w.S / dt, dt


def oracle_threads(w, table64, n_threads: int):
    """The same oracle on n_threads host cores: grid, then degrid of the gridded result.

    The oracle's C routines run unchanged, several at once from Python threads (the binding releases
    the GIL). Gridding: visibilities whose footprint rows lie wholly inside one of n_threads bands of
    grid rows are gridded by that band's thread straight into one shared grid (the bands are
    disjoint, so no two threads add to the same cell); the few that straddle a band edge are gridded
    afterwards by one thread. Degridding: disjoint slices of the visibilities, one per thread. The
    sums equal the single-thread oracle's up to the order of additions.
    Returns (grid, degridded values, skipped count, seconds).
    """
    import concurrent.futures as cf
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    cell, _, _ = oracle.indices(w.G, w.S, w.oversample, w.uv)
    h = (w.S - 1) // 2
    valid = cell[:, 1] >= 0
    lo = cell[:, 1] - h
    band = max(1, -(-w.G // n_threads))
    b0 = np.where(valid, lo // band, -1)
    inside = valid & ((lo + w.S - 1) // band == b0)
    g = np.zeros((w.npol, w.G, w.G), np.complex128)
    parts = [np.flatnonzero(inside & (b0 == b)) for b in range(n_threads)]
    rest = np.flatnonzero(~inside)

    def grid_part(idx):
        if idx.size:
            oracle.grid(w.G, w.S, w.oversample, w.uv[idx], w.vis[idx], w.weights[idx], table64, out=g)

    with cf.ThreadPoolExecutor(n_threads) as ex:
        list(ex.map(grid_part, parts))
    skipped = 0
    if rest.size:
        _, skipped = oracle.grid(w.G, w.S, w.oversample, w.uv[rest], w.vis[rest], w.weights[rest], table64, out=g)
    slices = np.array_split(np.arange(w.n_vis), n_threads)
    out = np.empty((w.n_vis, w.npol), np.complex128)

    def degrid_part(idx):
        if idx.size:
            out[idx] = oracle.degrid(w.G, w.S, w.oversample, w.uv[idx], g, table64)[0]

    with cf.ThreadPoolExecutor(n_threads) as ex:
        list(ex.map(degrid_part, slices))
    return g, out, skipped, time.perf_counter() - t0


def cpu_oracle_rate_threads(w, table64, n_threads: int):
    """vis-taps/s of grid + degrid of the whole batch by the oracle on n_threads host cores."""
    _, _, skipped, dt = oracle_threads(w, table64, n_threads)
    return 2 * (w.n_vis - skipped) * w.S * w.S / dt, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = synth.quad_pol()
    import oracle
    oracle.build()
    table64 = oracle.kb_table(w.S, w.oversample, w.beta).astype(np.float32).astype(np.float64)
    n_cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_oracle_rate_threads(synth.scaled_down(w, 20_000), table64, n_cores)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = cpu_oracle_rate_threads(w, table64, n_cores)
        rates.append(r)
        times.append(dt)
    value = float(np.mean(rates))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "the whole batch per step (warm-up steps use 20,000 visibilities)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_cores, "kind": "oracle",
                         "sample": f"all {w.n_vis} visibilities per step, grid + degrid, FP64, the unchanged oracle on "
                                   f"{n_cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_compression(gb, autotune, torch, dev, cfg_grid, cfg_degrid, steps, warmup, seed):
    """Grid + degrid step on the cored quad-pol workload with and without compression (Sec. 2.2).

    The compressed step is compress -> grid(merged) -> degrid(merged) -> expand to every original
    visibility: the same results as the plain step, up to rounding. Rates count ORIGINAL
    visibility-taps, so the two are directly comparable.
    """
    w = synth.cored_quad_pol(seed=seed)
    S2 = w.S * w.S
    stream = torch.cuda.current_stream()
    uv = torch.from_numpy(w.uv).to(dev)
    vis = torch.from_numpy(w.vis).to(dev)
    wt = torch.from_numpy(w.weights).to(dev)
    table = gb.grid_make_kernel_table(w.S, w.oversample, w.beta, device=dev)
    gplan = gb.Plan(w.G, w.S, w.oversample, w.npol, **autotune.plan_kwargs(cfg_grid))
    dplan = gb.Plan(w.G, w.S, w.oversample, w.npol, **autotune.plan_kwargs(cfg_degrid))
    g = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device=dev)
    vis_out = torch.empty((w.n_vis, w.npol), dtype=torch.complex64, device=dev)
    bufs = (torch.empty((w.n_vis, 2), dtype=torch.float64, device=dev),
            torch.empty((w.n_vis, w.npol), dtype=torch.complex64, device=dev),
            torch.empty(w.n_vis, dtype=torch.int64, device=dev), torch.zeros(1, dtype=torch.int64, device=dev))
    dc = torch.empty((w.n_vis, w.npol), dtype=torch.complex64, device=dev)
    gb.grid_compress(gplan, uv, vis, wt, out=bufs, sync=False)
    m = int(bufs[3].item())  # a deterministic function of the inputs; read once, outside the timed steps
    uv_c, vis_c, run_of = bufs[0][:m], bufs[1][:m], bufs[2]

    def plain(ev):
        g.zero_()
        ev[0].record(stream)
        gb.grid(gplan, uv, vis, wt, table, g)
        gb.degrid(dplan, uv, g, table, vis_out)
        ev[1].record(stream)

    def compressed(ev):
        g.zero_()
        ev[0].record(stream)
        gb.grid_compress(gplan, uv, vis, wt, out=bufs, sync=False)
        ev[2].record(stream)
        gb.grid(gplan, uv_c, vis_c, None, table, g)
        gb.degrid(dplan, uv_c, g, table, dc[:m])
        ev[3].record(stream)
        gb.degrid_expand(dplan, run_of, dc[:m], None, vis_out)
        ev[1].record(stream)

    def run(fn):
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(warmup + steps)]
        for ev in evs:
            fn(ev)
        torch.cuda.synchronize()
        evs = evs[warmup:]
        tot = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
        parts = None
        if fn is compressed:
            parts = (float(np.mean([e[0].elapsed_time(e[2]) for e in evs])),
                     float(np.mean([e[3].elapsed_time(e[1]) for e in evs])))
        return tot, parts

    t0, _ = run(plain)
    t1, (tc, te) = run(compressed)
    taps = 2.0 * w.n_vis * S2
    return {"workload": "cored quad-pol: G=2048 S=7 O=8 P=4, 48 antennas in a 300 m core + 16 out to 8 km, "
                        "2016 bl x 1024 t x 4 ch = 8,257,536 vis",
            "n_vis": w.n_vis, "n_compressed": m, "ratio": w.n_vis / m,
            "ms_per_step_uncompressed": t0, "ms_per_step_compressed": t1, "compress_ms": tc, "expand_ms": te,
            "value_uncompressed": taps / (t0 / 1e3), "value_compressed": taps / (t1 / 1e3),
            "unit": "original vis-taps/s (grid + degrid)"}


SWEEP_SHAPES = [(1, 1), (2, 1), (1, 2), (2, 2), (4, 1), (1, 4), (4, 2), (2, 4), (3, 3), (4, 4), (8, 1), (1, 8), (8, 2), (2, 8)]
SWEEP_WORK = [(128, 128), (256, 128), (1024, 256)]   # (visibilities per team chunk, threads per CTA)


def time_grid(gb, plan, uv, vis, wt, table, g, reps=3):
    """Median CUDA-event time (ms) of grid() after two warm-up calls; the grid is zeroed outside the timing."""
    import torch
    for _ in range(2):
        gb.grid(plan, uv, vis, wt, table, g)
    ms = []
    for _ in range(reps):
        g.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        gb.grid(plan, uv, vis, wt, table, g)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.median(ms))


def measure_sweep(gb, w, uv, vis, wt, table, g, n_valid, peak):
    """Sec. 5's central comparison on this workload: gridding time and FP32 FMA fraction for every
    built coarsening shape with Bu*Bv <= 16 (the paper's sweep), each at its fastest chunk length and
    CTA size among SWEEP_WORK (chunked schedule, global flushes)."""
    rows = []
    gpa = n_valid * w.S * w.S * w.npol
    for bu, bv in SWEEP_SHAPES:
        best = None
        for L, T in SWEEP_WORK:
            try:
                plan = gb.Plan(w.G, w.S, w.oversample, w.npol, Bu=bu, Bv=bv, vis_per_chunk=L, threads=T)
            except gb.GridderError:
                continue
            ms = time_grid(gb, plan, uv, vis, wt, table, g)
            plan.close()
            if best is None or ms < best[0]:
                best = (ms, L, T)
        if best is None:
            continue
        ms, L, T = best
        rows.append({"Bu": bu, "Bv": bv, "grid_ms": ms, "vis_per_chunk": L, "threads": T,
                     "grid_fma_frac": fma_fraction(gpa / (ms / 1e3), peak)})
    g.zero_()
    plain = next((r for r in rows if (r["Bu"], r["Bv"]) == (1, 1)), None)
    best = min(rows, key=lambda r: r["grid_ms"]) if rows else None
    return {"workload": "quad-pol (the bench workload), gridding only", "shapes": rows,
            "best": {k: best[k] for k in ("Bu", "Bv", "grid_ms", "grid_fma_frac")} if best else None,
            "gain_vs_1x1": (plain["grid_ms"] / best["grid_ms"]) if plain and best else None,
            "paper_context": "Sec. 5: coarsening gains of 1.9x (quad-pol) and 3.2x (single-pol) on a GTX 980"}


SINGLE_POL_CANDIDATES = [(2, 2, 256, 128), (4, 2, 256, 128), (2, 4, 256, 128), (4, 4, 256, 128), (3, 3, 256, 128),
                         (8, 2, 256, 128), (4, 2, 1024, 256), (4, 2, 128, 128)]


def measure_single_pol(gb, torch, dev, peak):
    """The single-polarization coarsening gain at throughput scale (Sec. 5 reports 3.2x on a GTX 980):
    the precision workload (G=4096, S=15, O=16, P=1, 16,711,680 visibilities, FP32) gridded by the plain
    Romein kernel (B=1, 1024 visibilities per team) and by the fastest coarsened configuration among
    SINGLE_POL_CANDIDATES, in the same run."""
    w = synth.precision_single_pol()
    uv = torch.from_numpy(w.uv).to(dev)
    vis = torch.from_numpy(w.vis).to(dev)
    wt = torch.from_numpy(w.weights).to(dev)
    table = gb.grid_make_kernel_table(w.S, w.oversample, w.beta, device=dev)
    g = torch.zeros((1, w.G, w.G), dtype=torch.complex64, device=dev)
    gpa = w.n_vis * w.S * w.S
    plain = gb.Plan(w.G, w.S, w.oversample, 1, B=1, vis_per_chunk=1024, schedule="chunked")
    p_ms = time_grid(gb, plain, uv, vis, wt, table, g)
    plain.close()
    best = None
    for bu, bv, L, T in SINGLE_POL_CANDIDATES:
        plan = gb.Plan(w.G, w.S, w.oversample, 1, Bu=bu, Bv=bv, vis_per_chunk=L, threads=T)
        ms = time_grid(gb, plan, uv, vis, wt, table, g)
        plan.close()
        if best is None or ms < best[0]:
            best = (ms, bu, bv, L, T)
    ms, bu, bv, L, T = best
    # degridding of the same workload: the sliding-window degridder and the tile gather in groups of 8
    out = torch.empty((w.n_vis, 1), dtype=torch.complex64, device=dev)
    degrid = {}
    for name, kw in (("chunked 4x4", dict(B=4, vis_per_chunk=64, threads=128)),
                     ("tile, groups of 8", dict(B=2, schedule="tile", threads=64, tile_group=8))):
        plan = gb.Plan(w.G, w.S, w.oversample, 1, **kw)
        degrid[name] = _event_ms(torch, lambda: gb.degrid(plan, uv, g, table, out))
        plan.close()
    del uv, vis, wt, g, out
    torch.cuda.empty_cache()
    return {"workload": "precision single-pol: G=4096 S=15 O=16 P=1, 256 antennas, 32,640 bl x 256 t x 2 ch = "
                        "16,711,680 vis, FP32", "plain_grid_ms": p_ms,
            "coarsened": {"Bu": bu, "Bv": bv, "vis_per_chunk": L, "threads": T, "grid_ms": ms},
            "degrid_ms": degrid,
            "gain": p_ms / ms, "plain_fma_frac": fma_fraction(gpa / (p_ms / 1e3), peak),
            "coarsened_fma_frac": fma_fraction(gpa / (ms / 1e3), peak),
            "paper_context": "Sec. 5: 3.2x single-pol coarsening gain on a GTX 980"}


def _event_ms(torch, fn, warmup=2, reps=5):
    """Median CUDA-event time of fn() on the current stream, after warm-up calls."""
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return sorted(ts)[len(ts) // 2]


def measure_small(gb, torch, dev):
    """The small single-pol case (G=256, S=7, O=8, P=1, 30,720 visibilities; launch latency dominates):
    the plain Romein gridder (B=1, 1024 visibilities per team), the coarsened one (2x2, 32 per team),
    and the sliding-window and tile degridders."""
    w = synth.plain_single_pol()
    uv = torch.from_numpy(w.uv).to(dev)
    vis = torch.from_numpy(w.vis).to(dev)
    wt = torch.from_numpy(w.weights).to(dev)
    table = gb.grid_make_kernel_table(w.S, w.oversample, w.beta, device=dev)
    g = torch.zeros((1, w.G, w.G), dtype=torch.complex64, device=dev)
    out = torch.empty((w.n_vis, 1), dtype=torch.complex64, device=dev)
    res = {"workload": "plain single-pol: G=256 S=7 O=8 P=1, 16 antennas, 120 bl x 256 t = 30,720 vis"}
    for name, kw, op in (("plain_grid_ms", dict(B=1, vis_per_chunk=1024), "grid"),
                         ("coarsened_grid_ms", dict(B=2, vis_per_chunk=32), "grid"),
                         ("degrid_ms", dict(B=2, vis_per_chunk=32), "degrid"),
                         ("tile_degrid_ms", dict(B=2, schedule="tile"), "degrid")):
        plan = gb.Plan(w.G, w.S, w.oversample, 1, **kw)
        if op == "grid":
            res[name] = _event_ms(torch, lambda: gb.grid(plan, uv, vis, wt, table, g))
        else:
            res[name] = _event_ms(torch, lambda: gb.degrid(plan, uv, g, table, out))
        plan.close()
    return res


def measure_batch(gb, torch, dev, peak):
    """The batching workload (64 channels x 8 w-planes = 512 single-pol grids of 1024^2, S by plane
    7, 7, 9, 9, 11, 11, 15, 15, 20,000,000 visibilities with uneven counts) in one persistent launch
    with 2x2 blocks."""
    ws = [w for row in synth.batched() for w in row]
    tables = {S: gb.grid_make_kernel_table(S, 8, 2.34 * S, device=dev) for S in sorted({w.S for w in ws})}
    items = [dict(uv=torch.from_numpy(w.uv).to(dev), vis=torch.from_numpy(w.vis).to(dev),
                  weights=torch.from_numpy(w.weights).to(dev), table=tables[w.S],
                  grid=torch.zeros((1, w.G, w.G), dtype=torch.complex64, device=dev), S=w.S) for w in ws]
    bp = gb.BatchPlan(1024, 8, 1, Bu=2, Bv=2, max_S=15)
    bp.set(items)
    ms = _event_ms(torch, bp.execute)
    gpa = float(sum(w.n_vis * w.S * w.S for w in ws))
    n = sum(w.n_vis for w in ws)
    del items, bp
    torch.cuda.empty_cache()
    return {"workload": f"batching: 512 single-pol grids of 1024^2 (64 channels x 8 w-planes, S by plane 7,7,9,9,11,11,15,15), "
                        f"{n:,} vis with uneven counts", "plan": "one persistent launch, 2x2 blocks",
            "grid_ms": ms, "vis_taps_per_s": gpa / (ms / 1e3), "fma_frac": fma_fraction(gpa / (ms / 1e3), peak)}


def measure_differentiation(gb, torch, dev, peak):
    """The differentiation workload (G=1024, S=7, O=8, P=1, 1,000,000 visibilities): the forward
    grid, the backward degrid_weighted (tile schedule), and one autograd step through both with an
    image-domain loss sum |IFFT(grid) - target|^2 (the FFT is PyTorch's)."""
    from paper_1605_07023_gb300.autograd import grid_op
    w = synth.differentiation()
    table = gb.grid_make_kernel_table(w.S, w.oversample, w.beta, device=dev)
    plan = gb.Plan(w.G, w.S, w.oversample, 1, B=2, schedule="tile")
    uv = torch.from_numpy(w.uv).to(dev)
    wt = torch.from_numpy(w.weights).to(dev)
    vis0 = torch.from_numpy(w.vis).to(dev)
    target = torch.from_numpy(synth.gaussian_sources_image(w.G, 5, seed=0)).to(dev).to(torch.complex64)
    g = torch.zeros((1, w.G, w.G), dtype=torch.complex64, device=dev)

    def fwd():
        g.zero_()
        gb.grid(plan, uv, vis0, wt, table, g)

    def bwd():
        gb.degrid_weighted(plan, uv, g, table, wt)

    def step():
        vis = vis0.clone().requires_grad_(True)
        img = torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(grid_op(plan, uv, vis, wt, table)[0]), norm="forward"))
        torch.sum(torch.abs(img - target) ** 2).backward()

    f_ms, b_ms, s_ms = _event_ms(torch, fwd), _event_ms(torch, bwd), _event_ms(torch, step)
    gpa = float(w.n_vis * w.S * w.S)
    plan.close()
    return {"workload": "differentiation: G=1024 S=7 O=8 P=1, 1,000,000 vis", "plan": "2x2 blocks, tile schedule",
            "grid_ms": f_ms, "degrid_weighted_ms": b_ms, "autograd_step_ms": s_ms,
            "grid_vis_taps_per_s": gpa / (f_ms / 1e3), "degrid_vis_taps_per_s": gpa / (b_ms / 1e3)}


def parse_cfg(s):
    """'schedule:Bu,Bv[:L[:T[:bin_u,bin_v | :group]]]' (L visibilities per chunk, T threads per CTA, bin
    sides in cells for the lazy schedule, visibilities per warp group for the tile schedule) -> plan
    config dict."""
    parts = s.split(":")
    bu, bv = (int(x) for x in parts[1].split(","))
    cfg = dict(schedule=parts[0], Bu=bu, Bv=bv)
    if len(parts) > 2:
        cfg["vis_per_chunk"] = int(parts[2])
    if len(parts) > 3:
        cfg["threads"] = int(parts[3])
    if len(parts) > 4 and parts[0] == "tile":
        cfg["tile_group"] = int(parts[4])
    elif len(parts) > 4:
        cfg["bin_u"], cfg["bin_v"] = (int(x) for x in parts[4].split(","))
    return cfg


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_1605_07023_gb300 as gb
    from paper_1605_07023_gb300 import autotune

    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # weak scaling: every rank grids its own observation (independent problems, different seed)
    from paper_1605_07023_gb300 import sharding
    w = synth.quad_pol(seed=sharding.rank_seed(0, rank))
    if args.vis:
        w = synth.scaled_down(w, args.vis)
    S2 = w.S * w.S
    stream = torch.cuda.current_stream()

    uv = torch.from_numpy(w.uv).to(dev)
    vis = torch.from_numpy(w.vis).to(dev)
    wt = torch.from_numpy(w.weights).to(dev)
    table = gb.grid_make_kernel_table(w.S, w.oversample, w.beta, device=dev)
    grid_buf = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device=dev)
    vis_out = torch.empty((w.n_vis, w.npol), dtype=torch.complex64, device=dev)
    torch.cuda.synchronize()

    # ---- choose the coarsened configuration (untimed)
    if args.config == "auto":
        best_grid = autotune.tune_grid(w, uv, vis, wt, table, grid_buf, reps=2)
    else:
        best_grid = parse_cfg(args.config)
    if args.degrid_config == "auto":
        best_degrid = autotune.tune_degrid(w, uv, table, grid_buf, vis_out, reps=2)
    else:
        best_degrid = parse_cfg(args.degrid_config)
    gplan = gb.Plan(w.G, w.S, w.oversample, w.npol, **autotune.plan_kwargs(best_grid))
    dplan = gb.Plan(w.G, w.S, w.oversample, w.npol, **autotune.plan_kwargs(best_degrid))
    pplan = gb.Plan(w.G, w.S, w.oversample, w.npol, B=1, vis_per_chunk=1024, schedule="chunked")

    def step(gp, dp, ev=None):
        grid_buf.zero_()
        if ev is not None:
            ev[0].record(stream)
        gb.grid(gp, uv, vis, wt, table, grid_buf)
        if ev is not None:
            ev[1].record(stream)
        gb.degrid(dp, uv, grid_buf, table, vis_out)
        if ev is not None:
            ev[2].record(stream)

    def timed(gp, dp, K, W):
        for _ in range(W):
            step(gp, dp)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
        barrier(world)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(K):
            step(gp, dp, evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        total_ms = t0.elapsed_time(t1)
        g_ms = [e[0].elapsed_time(e[1]) for e in evs]
        d_ms = [e[1].elapsed_time(e[2]) for e in evs]
        return total_ms, float(np.mean(g_ms)), float(np.mean(d_ms))

    gplan.skipped(reset=True)
    with ClockSampler(local) as clk:
        total_ms, g_ms, d_ms = timed(gplan, dplan, args.steps, args.warmup)
    n_skipped = gplan.skipped() // (args.steps + args.warmup)
    n_valid = w.n_vis - n_skipped
    total_ms = max_over_ranks(total_ms, world)
    ms_step = total_ms / args.steps
    taps_all = sum_over_ranks(2.0 * n_valid * S2, world)
    value = taps_all * args.steps / (total_ms / 1e3)

    # plain Romein (B=1, chunked, 1024 vis per team), same inputs
    if args.skip_plain:
        p_total, p_g, p_d = float("nan"), float("nan"), float("nan")
    else:
        p_total, p_g, p_d = timed(pplan, pplan, args.steps, args.warmup)
    p_value = 2.0 * n_valid * S2 / (p_total / args.steps / 1e3)

    sweep = single = batch = diff = small = None
    info = gb.device_info()
    clocks = clk.summary()
    max_mhz = clocks["sm_max_mhz"] or info["max_clock_khz"] / 1e3
    derived_peak = fma_peak_tflops(info["sm_count"], max_mhz)
    # the denominator: FP32 FMA throughput measured in this run by the library's own FFMA2 kernel
    peak = max(gb.measure_fma_peak(iters=32768) for _ in range(3))
    useful_flops = FLOPS_PER_GPA * n_valid * S2 * w.npol  # 2 FFMA (4 flop) per useful grid-point addition
    gpa_g = n_valid * S2 * w.npol / (g_ms / 1e3)
    gpa_d = n_valid * S2 * w.npol / (d_ms / 1e3)
    g_tflops = useful_flops / (g_ms / 1e3) / 1e12
    d_tflops = useful_flops / (d_ms / 1e3) / 1e12
    pg_tflops = useful_flops / (p_g / 1e3) / 1e12
    dominant = "grid" if g_ms >= d_ms else ("degrid_tile" if best_degrid["schedule"] == "tile" else "degrid")
    achieved = g_tflops if dominant == "grid" else d_tflops

    if not args.no_sweep and not args.vis:
        sweep = measure_sweep(gb, w, uv, vis, wt, table, grid_buf, n_valid, peak)
        single = measure_single_pol(gb, torch, dev, peak)
    if not args.no_extra and not args.vis:
        batch = measure_batch(gb, torch, dev, peak)
        diff = measure_differentiation(gb, torch, dev, peak)
        small = measure_small(gb, torch, dev)

    # DRAM bytes per launch from one ncu capture (profiles/traffic.json), used only while the
    # kernel's source file is the one that was captured
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    tkey = ("grid_" + best_grid["schedule"]) if dominant == "grid" else dominant
    if os.path.exists(tpath) and not args.vis:
        try:
            ent = json.load(open(tpath))["kernels"][tkey]
            files = ent["source"] if isinstance(ent["source"], list) else [ent["source"]]
            src = b"".join(open(os.path.join(ROOT, "paper_1605_07023_gb300", "csrc", f), "rb").read() for f in files)
            if hashlib.sha256(src).hexdigest()[:16] == ent["sha256_16"]:
                traffic = ent["bytes"]
        except Exception:
            traffic = None

    # ---- e2e through the C ABI from pinned host buffers: grid_degrid_host_steps() runs the timed steps
    # in one call; each step zeroes the grid, uploads uv, values and weights, grids, degrids and downloads
    # the grid and the degridded values. Copies overlap the kernels and the next step's uploads overlap
    # this step's downloads; every byte of every step crosses the link inside the timed region.
    e2e = None
    if not args.no_e2e:
        h_uv = torch.from_numpy(w.uv).pin_memory()
        h_vis = torch.from_numpy(w.vis).pin_memory()
        h_wt = torch.from_numpy(w.weights).pin_memory()
        h_grid = torch.empty((w.npol, w.G, w.G), dtype=torch.complex64).pin_memory()
        h_out = torch.empty((w.n_vis, w.npol), dtype=torch.complex64).pin_memory()
        h2d = h_uv.numel() * 8 + h_vis.numel() * 8 + h_wt.numel() * 4
        d2h = h_grid.numel() * 8 + h_out.numel() * 8
        work = [(uv, vis, wt, vis_out), (torch.empty_like(uv), torch.empty_like(vis), torch.empty_like(wt),
                                         torch.empty_like(vis_out))]

        def e2e_steps(k):
            # k passes in one call: step s+1's uploads overlap step s's degridding and downloads
            steps = [dict(uv=h_uv, vis=h_vis, weights=h_wt, vis_out=h_out, grid_out=h_grid) for _ in range(k)]
            gb.grid_degrid_host_steps(gplan, dplan, steps, table, grid_buf, work=work, stream=stream)

        e2e_steps(max(args.warmup, 1))
        barrier(world)
        torch.cuda.synchronize()
        t = time.perf_counter()
        e2e_steps(args.steps)
        torch.cuda.synchronize()
        et = max_over_ranks(time.perf_counter() - t, world)
        barrier(world)
        e2e = {"value": taps_all * args.steps / et, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * et / args.steps,
               "api": "grid_degrid_host_steps (C ABI, pinned host buffers; uploads, kernels and downloads overlapped within and across steps)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        table64 = oracle.kb_table(w.S, w.oversample, w.beta)
        # the whole batch, repeated until about 10 s of CPU work
        rates, spent = [], 0.0
        while spent < 10.0 and len(rates) < 4:
            r, dt = cpu_oracle_rate(w, w.n_vis, table64)
            rates.append(r)
            spent += dt
        one = {"value": float(np.mean(rates)), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"all {w.n_vis} visibilities x {len(rates)}, grid + degrid, FP64, 1 thread ({spent:.1f} s)"}
        n_cores = os.cpu_count() or 1
        prates, pspent = [], 0.0
        while pspent < 4.0 and len(prates) < 4:
            r, dt = cpu_oracle_rate_threads(w, table64, n_cores)
            prates.append(r)
            pspent += dt
        cpu = {"value": float(np.mean(prates)), "unit": UNIT, "cores": n_cores, "kind": "oracle",
               "sample": f"all {w.n_vis} visibilities x {len(prates)}, grid + degrid, FP64, the unchanged oracle "
                         f"on {n_cores} threads (gridding by disjoint bands of grid rows, degridding by disjoint "
                         f"slices) ({pspent:.1f} s)",
               "single_core": one}

    comp = None
    if not args.no_compression and not args.vis:
        comp = measure_compression(gb, autotune, torch, dev, best_grid, best_degrid, args.steps, args.warmup,
                                   sharding.rank_seed(0, rank))

    launches_per_step = (4 if best_grid["schedule"] == "patch" else 1) + 1
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded earth-rotation uv tracks, complex Gaussian values; stand-in for the paper's MeerKAT set)",
            "config": {"workload": WORKLOAD if not args.vis else f"{WORKLOAD}, cut to the first {w.n_vis:,}",
                       "grid_plan": best_grid, "degrid_plan": best_degrid,
                       "cache": "inputs (429 MB) larger than L2 (129 MB); grid zeroed inside each step",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "grid_ms": g_ms, "degrid_ms": d_ms,
            "grid_taps_per_s": n_valid * S2 / (g_ms / 1e3), "degrid_taps_per_s": n_valid * S2 / (d_ms / 1e3),
            "grid_fma_frac": fma_fraction(gpa_g, peak), "degrid_fma_frac": fma_fraction(gpa_d, peak),
            "grid_fma_frac_paper_counting": fma_fraction(gpa_g, peak, PAPER_FLOPS_PER_GPA),
            "plain": {"value": p_value, "unit": UNIT, "ms_per_step": p_total / args.steps, "grid_ms": p_g, "degrid_ms": p_d,
                      "grid_fma_frac": pg_tflops / peak,
                      "kernel": "Romein B=1 (chunked schedule, input order), 1024 vis per team, global-memory flushes"},
            "speedup_vs_plain": value / p_value, "grid_speedup_vs_plain": p_g / g_ms,
            "roofline": {"bound": "alu", "kernel": gplan.gridder() if dominant == "grid" else dominant,
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_note": "measured in this run: grid_measure_fma_peak (independent FFMA2 chains, 64 warps "
                                      f"per SM); derived {info['sm_count']} SMs x 128 FP32 FMA lanes x 2 flop x "
                                      f"{max_mhz:.0f} MHz = {derived_peak:.1f}; achieved counts 4 flop per useful "
                                      "grid-point addition (real taps), padding excluded"},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
            "n_valid_vis": n_valid,
        }
        if e2e is not None:
            line["e2e"] = e2e
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if comp is not None:
            line["compression"] = comp
        if sweep is not None:
            line["sweep"] = sweep
        if single is not None:
            line["single_pol"] = single
        if batch is not None:
            line["batch"] = batch
        if diff is not None:
            line["differentiation"] = diff
        if small is not None:
            line["small"] = small
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
