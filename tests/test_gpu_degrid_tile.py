"""Degridding with the tile schedule (one warp per 32 visibilities, footprints gathered from a
shared-memory copy of their bounding box) against the FP64 oracle.

Covers: every unrolled support S (odd, 1..15) and P in {1, 2, 4}; supports without an unrolled
kernel (even, or up to 64) through the run-time-support kernel; baseline-ordered tracks (the tile
path) and unordered positions (groups too large for the tile read the grid directly); CTA sizes
of 1 to 8 warps; weights (degrid_weighted); positions outside the valid region and non-finite
ones (skipped and zero, counted like the oracle); groups cut short by the end of the input; 16-bit
taps; unsupported shapes and CTA sizes rejected; the full 8,257,536-visibility quad-pol workload;
groups of 8 visibilities with four lanes each.
Tolerance: rel L2 <= 1e-5 per polarization.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1605_07023_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1605_07023_gb300 as gb
    return gb


@functools.lru_cache(maxsize=None)
def quad_pol():
    return synth.quad_pol()


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def kb32(S, O):
    return oracle.kb_table(S, O, 2.34 * S).astype(np.float32).astype(np.float64)


def random_grid(P, G, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((P, G, G)) + 1j * rng.standard_normal((P, G, G))).astype(np.complex64)


def check(gb, w, threads=0, weights=None, seed=0, precision="f32", group=0):
    # the plan also sets up gridding: 2x2 blocks make a team of more than 1024 threads above S=61
    B = 2 if w.S <= 40 else 4
    table = kb32(w.S, w.oversample)
    if precision != "f32":
        tdt = torch.bfloat16 if precision == "bf16" else torch.float16
        tab = torch.from_numpy(table).to(tdt).cuda()
        table = tab.float().cpu().numpy().astype(np.float64)
    else:
        tab = torch.from_numpy(table.astype(np.float32)).cuda()
    g = random_grid(w.npol, w.G, seed)
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, B=B, schedule="tile", threads=threads, precision=precision,
                   tile_group=group)
    uv = torch.from_numpy(np.ascontiguousarray(w.uv)).cuda()
    gd = torch.from_numpy(g).cuda()
    if weights is None:
        out = gb.degrid(plan, uv, gd, tab)
    else:
        out = gb.degrid_weighted(plan, uv, gd, tab, torch.from_numpy(weights).cuda())
    torch.cuda.synchronize()
    ref, skipped = oracle.degrid(w.G, w.S, w.oversample, w.uv, g.astype(np.complex128), table)
    if weights is not None:
        ref = ref * weights[:, None]
    got = out.cpu().numpy()
    assert plan.skipped() == skipped
    assert plan.status() == 0  # every bulk copy of a box completed
    for p in range(w.npol):
        e = rel_l2(got[:, p], ref[:, p])
        assert e <= TOL, (w.name, p, e)
    return got, ref


def track(S, O, P, n_times=96, seed=0):
    """Baseline-ordered tracks on a 256-cell grid with support S (the tile path)."""
    return synth.observation(f"tracks S{S} P{P}", 256, S, O, P, 12, 1000.0, n_times, 2, seed)


@pytest.mark.parametrize("S", [1, 3, 5, 7, 9, 11, 13, 15])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_every_support_tracks_and_random(gb, S, P):
    check(gb, track(S, 8, P, seed=S))
    check(gb, synth.random_uniform(128, S, 8, P, 4_003, seed=S + 10 * P))


@pytest.mark.parametrize("threads", [32, 64, 224, 256])
def test_cta_sizes(gb, threads):
    check(gb, synth.scaled_down(quad_pol(), 100_003), threads=threads)


def test_precision_workload_subset(gb):
    check(gb, synth.scaled_down(synth.precision_single_pol(), 300_000))


def test_weighted(gb):
    w = synth.scaled_down(quad_pol(), 60_001)
    rng = np.random.default_rng(3)
    check(gb, w, weights=rng.uniform(0.1, 3.0, w.n_vis).astype(np.float32))


@pytest.mark.parametrize("precision", ["bf16", "f16"])
def test_16bit_taps(gb, precision):
    check(gb, synth.scaled_down(quad_pol(), 40_000), precision=precision)


def test_invalid_and_edge_positions(gb):
    """Footprints touching every edge, positions just outside the valid region, inf and nan,
    mixed into groups with valid ones."""
    G, S, O = 64, 7, 8
    h = (S - 1) // 2
    lim = G / 2 - h
    rng = np.random.default_rng(5)
    pts = list(rng.uniform(-lim, lim - 1, size=(200, 2)))
    for a in (-lim, lim - 1, lim - 0.5, lim, -lim - 0.5, 0.0):
        for b in (-lim, lim - 1, 0.3, lim + 3):
            pts.append((a, b))
    pts += [(np.inf, 0.0), (0.0, np.nan), (-np.inf, 1.0), (1e300, 2.0)]
    uv = np.array(pts, dtype=np.float64)
    w = synth.Workload("edges", G, S, O, 2, uv, np.zeros((len(uv), 2), np.complex64), np.ones(len(uv), np.float32),
                       beta=2.34 * S)
    got, ref = check(gb, w)
    assert np.count_nonzero(got[np.all(ref == 0, axis=1)]) == 0


@pytest.mark.parametrize("G,S,P", [(16, 7, 1), (24, 7, 4), (32, 15, 2), (40, 9, 4)])
def test_small_grids(gb, G, S, P):
    """Grids not much larger than (or smaller than) a tile's box: the tensor copies reach past the
    right and bottom edges (zero fill), or the maps cannot be encoded and every group reads the grid
    directly; either way the same sums."""
    check(gb, synth.random_uniform(G, S, 8, P, 2_000, seed=G + S))


@pytest.mark.parametrize("n", [0, 1, 31, 33, 65])
def test_short_inputs(gb, n):
    base = synth.scaled_down(quad_pol(), 100)
    if n == 0:
        plan = gb.Plan(base.G, base.S, base.oversample, 4, B=2, schedule="tile")
        out = gb.degrid(plan, torch.zeros((0, 2), dtype=torch.float64, device="cuda"),
                        torch.zeros((4, base.G, base.G), dtype=torch.complex64, device="cuda"),
                        torch.from_numpy(kb32(base.S, base.oversample).astype(np.float32)).cuda())
        assert out.shape[0] == 0
        return
    check(gb, synth.scaled_down(quad_pol(), n))


@pytest.mark.parametrize("S,P", [(S, P) for P in (1, 4) for S in (2, 4, 8, 16, 17, 24, 31, 33, 48)] + [(64, 1)])
def test_run_time_supports(gb, S, P):
    """Supports without an unrolled kernel run the kernel that reads S from the plan and its taps
    from the shared-memory table; at S=48 and P=4 one warp's tile (137 KB) leaves room for one warp
    per CTA. (A plan also sets up gridding, whose teams limit S=64 to single polarization here.)"""
    check(gb, track(S, 8, P, seed=S))
    check(gb, synth.random_uniform(256, S, 8, P, 2_003, seed=S + 10 * P), threads=128)


@pytest.mark.parametrize("precision", ["bf16", "f16"])
def test_run_time_support_16bit_taps_and_weights(gb, precision):
    """The run-time-support kernel with 16-bit taps, and with weights (degrid_weighted)."""
    check(gb, track(10, 8, 4, seed=7), precision=precision)
    w = track(16, 16, 2, seed=8)
    rng = np.random.default_rng(9)
    check(gb, w, weights=rng.uniform(0.1, 3.0, w.n_vis).astype(np.float32), threads=64)


@pytest.mark.parametrize("G,S,P", [(20, 8, 4), (70, 64, 1), (96, 33, 2), (80, 48, 4)])
def test_run_time_supports_small_grids(gb, G, S, P):
    """The run-time-support kernel on grids close to (or smaller than) its box."""
    check(gb, synth.random_uniform(G, S, 8, P, 1_500, seed=G + S))


def test_unsupported_shapes_are_rejected(gb):
    for S, O, P, threads in [(7, 8, 4, 48), (7, 8, 4, 100), (60, 256, 4, 0)]:
        # CTAs of a part of a warp; a tile (173 KB) and table (61 KB) that do not fit together
        with pytest.raises(gb.GridderError) as e:
            gb.Plan(256, S, O, P, B=4, schedule="tile", threads=threads)
        assert e.value.code in (-1, -2)


def test_tile_plan_grids_like_chunked(gb):
    """A tile plan grids with the chunked kernel."""
    w = synth.scaled_down(quad_pol(), 80_000)
    table = kb32(w.S, w.oversample)
    plan = gb.Plan(w.G, w.S, w.oversample, 4, B=2, schedule="tile")
    g = torch.zeros((4, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, torch.from_numpy(w.uv).cuda(), torch.from_numpy(w.vis).cuda(), None,
            torch.from_numpy(table.astype(np.float32)).cuda(), g)
    torch.cuda.synchronize()
    ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, None, table)
    for p in range(4):
        assert rel_l2(g.cpu().numpy()[p], ref[p]) <= TOL


def test_full_quad_pol(gb):
    """All 8,257,536 visibilities with the tile schedule at 1, 2 and 4 warps per CTA, and in groups
    of 8."""
    w = quad_pol()
    check(gb, w, threads=32)
    check(gb, w, threads=64, seed=1)
    check(gb, w, threads=128, seed=2)
    check(gb, w, threads=128, seed=3, group=8)


@pytest.mark.parametrize("S", [1, 3, 7, 15, 2, 8, 16, 33])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_groups_of_8(gb, S, P):
    """Groups of 8 visibilities, four lanes per visibility (each summing every fourth footprint row,
    the partial sums added by shuffles), with unrolled and run-time supports, on tracks and on
    unordered positions."""
    check(gb, track(S, 8, P, seed=S), group=8)
    check(gb, synth.random_uniform(256, S, 8, P, 2_003, seed=S + 10 * P), threads=64, group=8)


def test_groups_of_8_fast_tracks(gb):
    """The precision workload's first 300,000 visibilities (tracks that move several cells per
    visibility) in groups of 8, with weights and with 16-bit taps; and inputs that end inside a
    group."""
    w = synth.scaled_down(synth.precision_single_pol(), 300_000)
    check(gb, w, group=8)
    rng = np.random.default_rng(4)
    check(gb, w, weights=rng.uniform(0.1, 3.0, w.n_vis).astype(np.float32), threads=32, group=8)
    check(gb, synth.scaled_down(quad_pol(), 40_000), precision="bf16", group=8)
    for n in (1, 7, 9, 33):
        check(gb, synth.scaled_down(quad_pol(), n), group=8)
