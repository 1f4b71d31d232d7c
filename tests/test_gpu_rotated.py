"""The sorted schedule's gridder (box-ordered batches, rotated tap tables, staged move masks) against
the FP64 oracle, through the C ABI, on inputs chosen to stress its reordering and its move masks.

Bar: relative L2 error <= 1e-5 per polarization plane, and the oracle's count of skipped
visibilities. Which kernel a plan launches is checked through grid_plan_gridder().
"""
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


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def kb32(S, O):
    return oracle.kb_table(S, O, 2.34 * S).astype(np.float32).astype(np.float64)


def check(gb, w, Bu, Bv, expect=None, **kw):
    table32 = kb32(w.S, w.oversample)
    kw.setdefault("schedule", "sorted")
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, Bu=Bu, Bv=Bv, **kw)
    if expect is not None:
        assert plan.gridder() == expect
    uv = torch.from_numpy(np.ascontiguousarray(w.uv)).cuda()
    vis = torch.from_numpy(np.ascontiguousarray(w.vis)).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w.weights)).cuda()
    tab = torch.from_numpy(table32.astype(np.float32)).cuda()
    g = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, uv, vis, wt, tab, g)
    torch.cuda.synchronize()
    got = g.cpu().numpy()
    ref, sk = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, table32)
    assert plan.skipped() == sk
    for p in range(w.npol):
        e = rel_l2(got[p], ref[p])
        assert e <= TOL, (Bu, Bv, kw, p, e)
    return plan


def tracks(n, G, S, seed, npol=4, speed=0.7, jitter=1.5):
    """Baseline-like tracks: slow drifts with channel-like back-and-forth steps of `jitter` cells."""
    rng = np.random.default_rng(seed)
    h = (S - 1) // 2
    lim = G / 2 - h - 2
    n_tr = max(1, n // 256)
    out = []
    for _ in range(n_tr):
        p0 = rng.uniform(-lim * 0.8, lim * 0.8, 2)
        ang = rng.uniform(0, 2 * np.pi)
        t = np.arange(256)
        base = p0 + np.outer(t // 4 * speed, [np.cos(ang), np.sin(ang)])
        ch = (t % 4)[:, None] * jitter / 3 * np.array([np.cos(ang + 1), np.sin(ang + 1)])
        out.append(np.clip(base + ch, -lim, lim))
    uv = np.concatenate(out)[:n]
    vis = (rng.standard_normal((len(uv), npol)) + 1j * rng.standard_normal((len(uv), npol))).astype(np.complex64)
    return synth.Workload("tracks", G, S, 8, npol, uv, vis, rng.uniform(0.5, 1.5, len(uv)).astype(np.float32))


def test_kernel_selection(gb):
    """Sorted plans run the narrow kernel for teams of up to 32 threads and the wide one up to 64;
    larger teams are refused. The other schedules keep their own kernels."""
    assert gb.Plan(2048, 7, 8, 4, B=2, vis_per_chunk=128, threads=128, schedule="sorted").gridder() == "sorted"
    assert gb.Plan(2048, 7, 8, 4, B=1, schedule="sorted").gridder() == "sorted-wide"          # 7 x 7 = 49
    assert gb.Plan(4096, 15, 16, 1, B=2, schedule="sorted").gridder() == "sorted-wide"        # 8 x 8 = 64
    assert gb.Plan(4096, 15, 16, 1, B=4, schedule="sorted").gridder() == "sorted"             # 5 x 5
    with pytest.raises(gb.GridderError) as e:
        gb.Plan(4096, 15, 16, 1, B=1, schedule="sorted")                                     # 225 threads
    assert e.value.code == -2
    assert gb.Plan(2048, 7, 8, 4, B=2).gridder() == "chunked"
    assert gb.Plan(2048, 7, 8, 4, B=2, schedule="patch").gridder() == "patch"
    assert gb.Plan(2048, 7, 8, 4, B=2, schedule="tile").gridder() == "chunked"


@pytest.mark.parametrize("Bu,Bv", [(2, 2), (1, 1), (2, 1), (4, 2), (3, 3), (4, 4), (8, 2), (1, 8)])
@pytest.mark.parametrize("npol", [1, 4])
def test_jittered_tracks(gb, Bu, Bv, npol):
    """Tracks that step back and forth across block edges (the case box ordering targets)."""
    w = tracks(40_000, 512, 7, seed=Bu * 7 + Bv + npol, npol=npol)
    check(gb, w, Bu, Bv)


@pytest.mark.parametrize("chunk", [1, 5, 31, 32, 33, 64, 100, 128, 1000])
@pytest.mark.parametrize("threads", [32, 128, 256])
def test_chunk_lengths_and_ctas(gb, chunk, threads):
    """Chunks that end inside a batch or at its edge, and CTAs of one to sixteen teams."""
    w = tracks(20_011, 256, 7, seed=chunk + threads, npol=4)
    check(gb, w, 2, 2, "sorted", vis_per_chunk=chunk, threads=threads)


@pytest.mark.parametrize("order", ["reversed", "shuffled", "duplicates", "alternating"])
def test_orders(gb, order):
    """Input orders with no coherence, with many visibilities on one fine position (ties in the
    sort), and with the box jumping between two far positions every visibility."""
    w = tracks(30_000, 512, 7, seed=11, npol=4)
    rng = np.random.default_rng(2)
    if order == "reversed":
        w.uv = w.uv[::-1].copy()
    elif order == "shuffled":
        w.uv = w.uv[rng.permutation(len(w.uv))].copy()
    elif order == "duplicates":
        w.uv = np.repeat(w.uv[: len(w.uv) // 8], 8, axis=0)[: len(w.uv)].copy()
    else:
        w.uv[0::2] = [10.25, -20.5]
        w.uv[1::2] = [-100.0, 100.125]
    for B in [(2, 2), (1, 1), (4, 4)]:
        check(gb, w, *B)


def test_invalid_records_inside_batches(gb):
    """Invalid and off-grid visibilities at the start of chunks, inside batches, filling whole
    batches (the previous valid box must carry across them), and at the end of the data."""
    w = tracks(8_192, 256, 7, seed=5, npol=4)
    uv = w.uv.copy()
    bad = [np.nan, 1e9, -1e9, np.inf]
    idx = np.r_[0:3, 40, 41, 77, 128:160, 200:230, 256:320, 500, 1023, 1024, 1025, 4096:4224, 8000:8192]
    for k, i in enumerate(idx):
        uv[i] = [bad[k % 4], 0.0] if k % 2 else [0.0, bad[k % 4]]
    w.uv = uv
    for chunk in (32, 128, 1024):
        for B in [(2, 2), (1, 1), (3, 3)]:
            check(gb, w, *B, vis_per_chunk=chunk)


def test_edges_of_the_grid(gb):
    """Footprints on every edge and corner of the grid, for narrow and wide teams."""
    G, S = 64, 7
    h = 3
    lo, hi = h - G // 2, G // 2 - h - 1
    rng = np.random.default_rng(8)
    pts = rng.choice([lo, lo + 0.4, hi - 0.4, hi], size=(5000, 2))
    pts += rng.uniform(-0.3, 0.3, pts.shape) * (rng.random(pts.shape) < 0.5)
    pts = np.clip(pts, lo - 0.49, hi + 0.49)
    vis = (rng.standard_normal((5000, 2)) + 1j * rng.standard_normal((5000, 2))).astype(np.complex64)
    w = synth.Workload("corners", G, S, 8, 2, pts, vis, np.ones(5000, np.float32))
    for B in [(2, 2), (1, 1), (8, 2), (2, 8), (3, 3)]:
        check(gb, w, *B)


def test_sort_key_wraps_on_large_grids(gb):
    """Block indices above 2^13 (G = 10240, B = 1) wrap in the sort key; only the order changes."""
    G, S = 10240, 7
    rng = np.random.default_rng(4)
    base = np.array([4900.0, -4900.0])
    uv = base + np.cumsum(rng.uniform(-0.8, 0.8, (3000, 2)), axis=0) * 0.3
    uv = np.concatenate([uv, -uv, uv * [1, -1]])
    vis = (rng.standard_normal((len(uv), 1)) + 1j * rng.standard_normal((len(uv), 1))).astype(np.complex64)
    w = synth.Workload("far", G, S, 8, 1, uv, vis, np.ones(len(uv), np.float32))
    check(gb, w, 1, 1, "sorted-wide")
    check(gb, w, 2, 2, "sorted")


@pytest.mark.parametrize("precision", ["bf16", "f16"])
def test_16bit_storage(gb, precision):
    """16-bit values and taps through the rotated tables (rounded inputs on both sides)."""
    w = tracks(20_000, 512, 7, seed=3, npol=4)
    dt = torch.bfloat16 if precision == "bf16" else torch.float16
    table = torch.from_numpy(kb32(w.S, w.oversample).astype(np.float32)).to(dt)
    vis16 = torch.view_as_real(torch.from_numpy(w.vis)).to(dt)
    tab64 = table.float().double().numpy()
    vis_r = torch.view_as_complex(vis16.float().contiguous()).numpy().astype(np.complex128)
    plan = gb.Plan(w.G, w.S, w.oversample, 4, B=2, precision=precision, schedule="sorted")
    assert plan.gridder() == "sorted"
    g = torch.zeros((4, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, torch.from_numpy(w.uv).cuda(), vis16.cuda(), torch.from_numpy(w.weights).cuda(), table.cuda(), g)
    torch.cuda.synchronize()
    ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, vis_r, w.weights, tab64)
    got = g.cpu().numpy()
    for p in range(4):
        assert rel_l2(got[p], ref[p]) <= TOL


def test_full_quad_pol_sorted(gb):
    """All 8,257,536 visibilities of the quad-pol workload with the plan the benchmark tunes to (2x2
    blocks, 128 visibilities per chunk, 128-thread CTAs)."""
    check(gb, synth.quad_pol(), 2, 2, "sorted", vis_per_chunk=128, threads=128)


@pytest.mark.parametrize("B", [(2, 2), (4, 4), (8, 2)])
def test_precision_workload_subset_sorted(gb, B):
    """S=15, O=16, G=4096 single polarization (the precision workload's first 1,000,000
    visibilities): teams of 64 (2x2, the wide kernel), 25 (4x4) and 24 (8x2) threads with large
    rotated tables."""
    w = synth.scaled_down(synth.precision_single_pol(), 1_000_000)
    check(gb, w, *B, vis_per_chunk=256)
