"""Autotuner for the coarsening factors, schedule and chunk length.

Following Sec. 4: the best combination cannot be derived in closed form, so a
synthetic dataset is gridded with a range of coarsening factors and work
shapes, and the fastest is remembered. Tuning is separate per number of
polarizations (and per GCF size, grid and storage precision). Sec. 6 notes
that only near-square blocks (1:1 or 2:1) need trying; the candidate list
follows that.

Results are cached as JSON, keyed by GPU name and problem, in
$GB300_GRIDDER_CACHE (default ~/.cache/gb300_gridder/tune.json).
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import synth

BLOCK_CANDIDATES = [(1, 1), (2, 1), (1, 2), (2, 2), (4, 2), (2, 4), (3, 3), (4, 4), (8, 2), (2, 8)]
CHUNKED_LENGTHS = (128, 256, 1024)
PATCH_LENGTHS = (32, 64)
# Gridding schedules tried by default. The patch schedule measured about 5x slower than the chunked
# one on GB300 (the L2 atomics it saves are not what bounds the chunked kernel), so it is tried only
# when asked for (tune_grid(..., schedules=GRID_SCHEDULES + ("patch",))).
GRID_SCHEDULES = ("chunked", "sorted", "lazy")
# Sorted-schedule candidates: the shapes whose teams have at most 64 threads at small S are tried with
# the chunked lengths and CTA sizes; plan creation refuses the others.
# Lazy-box candidates: block shapes, with the default widened bin, one chunk length and CTA size.
LAZY_SHAPES = [(4, 2), (2, 4), (4, 4), (8, 4), (4, 8)]
DEGRID_LENGTHS = (64, 128, 256)
# Target CTA sizes (threads per CTA, rounded down to whole teams). Smaller CTAs let more of the
# register-limited teams be resident per SM.
CTA_THREADS = (128, 256)
TILE_THREADS = (32, 64, 128)   # tile-schedule degridding: warps per CTA x 32
TILE_GROUPS = (32, 8)          # tile-schedule degridding: visibilities per warp group


def _cache_path() -> str:
    return os.environ.get("GB300_GRIDDER_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gb300_gridder",
                                                               "tune.json"))


def _key(kind: str, G: int, S: int, O: int, P: int, precision: str) -> str:
    """Cache key: device, problem, and the candidate lists (a result tuned over other candidates,
    for example before a schedule existed, is not reused)."""
    import hashlib
    import torch
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    cands = repr((BLOCK_CANDIDATES, CHUNKED_LENGTHS, PATCH_LENGTHS, DEGRID_LENGTHS, CTA_THREADS, TILE_THREADS, GRID_SCHEDULES,
                  LAZY_SHAPES))
    return f"{name}|{kind}|G{G}|S{S}|O{O}|P{P}|{precision}|{hashlib.sha256(cands.encode()).hexdigest()[:8]}"


def load_cache() -> dict:
    try:
        with open(_cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(c: dict) -> None:
    p = _cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(c, fh, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def plan_kwargs(cfg: dict) -> dict:
    return dict(Bu=cfg["Bu"], Bv=cfg["Bv"], schedule=cfg["schedule"], vis_per_chunk=cfg.get("vis_per_chunk", 0),
                threads=cfg.get("threads", 0), precision=cfg.get("precision", "f32"), bin_u=cfg.get("bin_u", 0),
                bin_v=cfg.get("bin_v", 0), tile_group=cfg.get("tile_group", 0))


def _candidates(kind: str, schedules=GRID_SCHEDULES):
    for bu, bv in BLOCK_CANDIDATES:
        if kind == "grid":
            for sched in ("chunked", "sorted"):
                if sched in schedules:
                    for L in CHUNKED_LENGTHS:
                        for T in CTA_THREADS:
                            yield dict(schedule=sched, Bu=bu, Bv=bv, vis_per_chunk=L, threads=T)
            if "patch" in schedules:
                for L in PATCH_LENGTHS:
                    yield dict(schedule="patch", Bu=bu, Bv=bv, vis_per_chunk=L)
        else:
            for L in DEGRID_LENGTHS:
                for T in CTA_THREADS:
                    yield dict(schedule="chunked", Bu=bu, Bv=bv, vis_per_chunk=L, threads=T)
    if kind == "grid" and "lazy" in schedules:
        for bu, bv in LAZY_SHAPES:
            yield dict(schedule="lazy", Bu=bu, Bv=bv, vis_per_chunk=256, threads=128)
    if kind == "degrid":
        # the tile schedule does not use Bu, Bv or the chunk length for degridding; groups of 8
        # visibilities (four lanes each) are for tracks too fast for groups of 32
        for group in TILE_GROUPS:
            for T in TILE_THREADS:
                yield dict(schedule="tile", Bu=2, Bv=2, vis_per_chunk=0, threads=T, tile_group=group)


def _time(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_grid(w, uv, vis, wt, table, grid_buf, reps: int = 2, precision: str = "f32", verbose: bool = False,
              schedules=GRID_SCHEDULES) -> dict:
    """Fastest gridding configuration for these device inputs (each candidate is timed reps times)."""
    from . import Plan, grid, GridderError
    best, best_ms = None, float("inf")
    for cfg in _candidates("grid", schedules):
        try:
            plan = Plan(w.G, w.S, w.oversample, w.npol, precision=precision, **{k: v for k, v in plan_kwargs(cfg).items()
                                                                                   if k != "precision"})
        except GridderError:
            continue
        ms = _time(lambda: grid(plan, uv, vis, wt, table, grid_buf), reps)
        if verbose:
            print(f"grid {cfg}: {ms:.3f} ms", flush=True)
        if ms < best_ms:
            best, best_ms = dict(cfg, ms=ms), ms
        plan.close()
    grid_buf.zero_()
    return best


def tune_degrid(w, uv, table, grid_buf, vis_out, reps: int = 2, precision: str = "f32", verbose: bool = False) -> dict:
    from . import Plan, degrid, GridderError
    best, best_ms = None, float("inf")
    for cfg in _candidates("degrid"):
        try:
            plan = Plan(w.G, w.S, w.oversample, w.npol, precision=precision, **{k: v for k, v in plan_kwargs(cfg).items()
                                                                                   if k != "precision"})
        except GridderError:
            continue
        ms = _time(lambda: degrid(plan, uv, grid_buf, table, vis_out), reps)
        if verbose:
            print(f"degrid {cfg}: {ms:.3f} ms", flush=True)
        if ms < best_ms:
            best, best_ms = dict(cfg, ms=ms), ms
        plan.close()
    return best


def tune(G: int, S: int, oversample: int, npol: int, precision: str = "f32", n_vis: int = 1_000_000,
         use_cache: bool = True, verbose: bool = False) -> dict:
    """Tune on a small synthetic observation shaped like the problem; return {"grid": cfg, "degrid": cfg}.

    The dataset is a baseline-ordered earth-rotation observation (see synth) scaled to the grid.
    """
    import torch
    from . import grid_make_kernel_table
    key = _key("both", G, S, oversample, npol, precision)
    cache = load_cache() if use_cache else {}
    if key in cache:
        return cache[key]
    n_times = max(16, min(1024, n_vis // (2016 * 2)))
    w = synth.observation("tune", G, S, oversample, npol, 64, 4000.0, n_times, 2, seed=1234, limit=n_vis)
    dev = torch.device("cuda")
    uv = torch.from_numpy(w.uv).to(dev)
    if precision == "f32":
        vis = torch.from_numpy(w.vis).to(dev)
    else:
        dt = torch.bfloat16 if precision == "bf16" else torch.float16
        vis = torch.view_as_real(torch.from_numpy(w.vis)).to(dt).contiguous().to(dev)
    wt = torch.from_numpy(w.weights).to(dev)
    table = grid_make_kernel_table(S, oversample, 2.34 * S, precision)
    g = torch.zeros((npol, G, G), dtype=torch.complex64, device=dev)
    out = torch.empty((w.n_vis, npol), dtype=torch.complex64, device=dev)
    res = {"grid": tune_grid(w, uv, vis, wt, table, g, precision=precision, verbose=verbose),
           "degrid": tune_degrid(w, uv, table, g, out, precision=precision, verbose=verbose)}
    if use_cache:
        cache = load_cache()
        cache[key] = res
        save_cache(cache)
    return res


# Batched gridding: one-shape kernels and the two-shape pairs the library builds
BATCH_SHAPES = {1: [(1, 1), (2, 1), (1, 2), (2, 2), (3, 3), (4, 2), (2, 4), (4, 4)],
                4: [(1, 1), (2, 1), (2, 2), (4, 2)]}
BATCH_PAIRS = {1: [((2, 2), (4, 2)), ((2, 2), (2, 4)), ((2, 2), (4, 4)), ((2, 1), (2, 2)), ((2, 1), (4, 2))],
               4: [((2, 2), (4, 2)), ((2, 1), (2, 2))]}
BATCH_SPLITS = (9, 11, 13)


def tune_batch(G: int, oversample: int, npol: int, items, max_S: int, precision: str = "f32", reps: int = 2,
               verbose: bool = False) -> dict:
    """Fastest BatchPlan configuration for these items (each candidate set() and executed reps times).

    Candidates: every one-shape kernel, and every two-shape pair with S_split in BATCH_SPLITS (only splits
    that separate the items' supports). Returns the BatchPlan keyword arguments plus "ms". The items' grids
    are left holding gridded data; zero them before use.
    """
    from . import BatchPlan, GridderError
    supports = sorted({int(it["S"]) for it in items})
    cands = [dict(Bu=bu, Bv=bv) for bu, bv in BATCH_SHAPES.get(npol, [])]
    for (a, b) in BATCH_PAIRS.get(npol, []):
        for split in BATCH_SPLITS:
            if supports and supports[0] < split <= supports[-1]:
                cands.append(dict(Bu=a[0], Bv=a[1], Bu2=b[0], Bv2=b[1], S_split=split))
    best, best_ms = None, float("inf")
    for cfg in cands:
        try:
            bp = BatchPlan(G, oversample, npol, max_S=max_S, precision=precision, **cfg)
            bp.set(items)
        except GridderError:
            continue
        ms = _time(bp.execute, reps)
        if verbose:
            print(f"batch {cfg}: {ms:.3f} ms", flush=True)
        if ms < best_ms:
            best, best_ms = dict(cfg, ms=ms), ms
        bp.close()
    return best
