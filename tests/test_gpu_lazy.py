"""The lazy-box gridder (a bin wider than Sec. 3's, box moved only when the footprint leaves it)
against the FP64 oracle, through the C ABI.

Bar: relative L2 error <= 1e-5 per polarization plane (FP32 accumulation against FP64), and the
same skipped count as the oracle. The bin width changes only which thread adds which product, so
every shape and bin must give the oracle's sums.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1605_07023_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5

SHAPES = {1: [(2, 2), (4, 2), (2, 4), (4, 4), (8, 2), (2, 8), (8, 4), (4, 8), (8, 8)],
          2: [(2, 2), (4, 2), (2, 4), (4, 4), (8, 2), (2, 8)],
          4: [(2, 1), (2, 2), (4, 1), (4, 2), (2, 4), (8, 1)]}


@functools.lru_cache(maxsize=1)
def quad_pol():
    return synth.quad_pol()


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1605_07023_gb300 as gb
    return gb


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


def kb32(S, O):
    return oracle.kb_table(S, O, 2.34 * S).astype(np.float32).astype(np.float64)


def min_bin(S, B):
    return -(-(S + B - 1) // B) * B


def grid_gpu(gb, w, plan, table32):
    uv = torch.from_numpy(np.ascontiguousarray(w.uv)).cuda()
    vis = torch.from_numpy(np.ascontiguousarray(w.vis)).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w.weights)).cuda()
    tab = torch.from_numpy(table32.astype(np.float32)).cuda()
    g = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, uv, vis, wt, tab, g)
    torch.cuda.synchronize()
    return g.cpu().numpy()


def check(gb, w, Bu, Bv, ref=None, **kw):
    table32 = kb32(w.S, w.oversample)
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, Bu=Bu, Bv=Bv, schedule="lazy", **kw)
    got = grid_gpu(gb, w, plan, table32)
    if ref is None:
        ref = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, table32)
    g_ref, sk = ref
    assert plan.skipped() == sk
    for p in range(w.npol):
        e = rel_l2(got[p], g_ref[p])
        assert e <= TOL, (Bu, Bv, kw, p, e)
    return plan


def oracle_ref(w):
    t = kb32(w.S, w.oversample)
    return oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, t)


@pytest.mark.parametrize("Bu,Bv", SHAPES[1])
@pytest.mark.parametrize("slack", [0, 1, 2])
def test_lazy_plain_single_pol(gb, Bu, Bv, slack):
    """The 30,720-visibility G=256 single-pol workload, every built P=1 shape, bins of the paper's
    width and one or two blocks wider per axis (teams of at most 32 threads)."""
    w = synth.plain_single_pol()
    bu, bv = min_bin(w.S, Bu) + slack * Bu, min_bin(w.S, Bv) + slack * Bv
    if (bu // Bu) * (bv // Bv) > 32:
        pytest.skip("team wider than a warp")
    check(gb, w, Bu, Bv, ref=_plain_ref(), bin_u=bu, bin_v=bv)


@functools.lru_cache(maxsize=1)
def _plain_ref():
    return oracle_ref(synth.plain_single_pol())


@functools.lru_cache(maxsize=1)
def _quad_sub():
    w = synth.scaled_down(quad_pol(), 200_001)
    return w, oracle_ref(w)


@pytest.mark.parametrize("Bu,Bv", SHAPES[4])
def test_lazy_quad_pol_subset(gb, Bu, Bv):
    """The first 200,001 visibilities of the quad-pol G=2048 workload (a ragged tail), the default
    bin (one block of slack per axis) where the team fits a warp, else the paper's bin."""
    w, ref = _quad_sub()
    bu, bv = min_bin(w.S, Bu) + Bu, min_bin(w.S, Bv) + Bv
    if (bu // Bu) * (bv // Bv) > 32:
        bu, bv = min_bin(w.S, Bu), min_bin(w.S, Bv)
    check(gb, w, Bu, Bv, ref=ref, bin_u=bu, bin_v=bv)


@pytest.mark.parametrize("bins", [(12, 10), (12, 8), (16, 10), (12, 12), (16, 14), (20, 10)])
def test_lazy_quad_pol_4x2_bins(gb, bins):
    """4x2 blocks at P=4 with several bin widths (3x4 up to 5x5 blocks)."""
    w, ref = _quad_sub()
    check(gb, w, 4, 2, ref=ref, bin_u=bins[0], bin_v=bins[1])


@pytest.mark.parametrize("npol", [1, 2, 4])
def test_lazy_random_positions_and_weights(gb, npol):
    """Unordered positions (the box moves at almost every record), non-unit weights, every P."""
    w = synth.random_uniform(300, 9, 8, npol, 50_003, seed=npol)
    w.weights = np.random.default_rng(3).uniform(0.1, 2.0, w.n_vis).astype(np.float32)
    ref = oracle_ref(w)
    for Bu, Bv, bu, bv in [(2, 2, 10, 10), (4, 2, 16, 12), (4, 2, 12, 10)]:
        check(gb, w, Bu, Bv, ref=ref, bin_u=bu, bin_v=bv)


@pytest.mark.parametrize("chunk", [1, 7, 31, 32, 33, 512, 5000])
@pytest.mark.parametrize("threads", [32, 128, 256])
def test_lazy_chunk_lengths_and_cta_sizes(gb, chunk, threads):
    w = synth.scaled_down(quad_pol(), 40_000)
    check(gb, w, 4, 2, ref=_quad40k(), vis_per_chunk=chunk, threads=threads, bin_u=12, bin_v=10)


@functools.lru_cache(maxsize=1)
def _quad40k():
    return oracle_ref(synth.scaled_down(quad_pol(), 40_000))


def test_lazy_large_support(gb):
    """S=15, O=16 (the precision workload's kernel) on a subset, several P=1 shapes and bins."""
    w = synth.scaled_down(synth.precision_single_pol(), 100_000)
    ref = oracle_ref(w)
    for Bu, Bv, bu, bv in [(4, 4, 20, 20), (4, 4, 24, 20), (8, 2, 24, 18), (2, 8, 18, 24), (8, 2, 32, 16), (4, 4, 20, 24),
                           (8, 4, 24, 20), (4, 8, 20, 24), (8, 8, 24, 24), (8, 8, 32, 24)]:
        check(gb, w, Bu, Bv, ref=ref, bin_u=bu, bin_v=bv)


def test_lazy_edges_and_invalid(gb):
    """Footprints touching every grid edge (boxes reaching past the far edges), plus invalid and
    off-grid visibilities."""
    G, S, O = 64, 7, 8
    h = 3
    lo, hi = h - G // 2, G // 2 - h - 1
    rng = np.random.default_rng(5)
    pts = [[lo, lo], [hi, hi], [lo, hi], [hi, lo], [lo - 0.5, 0], [hi + 0.49, 0.2], [0, hi + 0.5], [np.nan, 0],
           [0, np.inf], [1e9, 0], [-40, 0]]
    uv = np.concatenate([np.array(pts, float), rng.uniform(lo - 2, hi + 2, (3000, 2))])
    vis = (rng.standard_normal((len(uv), 4)) + 1j * rng.standard_normal((len(uv), 4))).astype(np.complex64)
    w = synth.Workload("edges", G, S, O, 4, uv, vis, np.ones(len(uv), np.float32))
    ref = oracle_ref(w)
    for Bu, Bv, bu, bv in [(2, 2, 8, 8), (2, 2, 10, 10), (4, 2, 12, 10), (4, 2, 16, 12), (8, 1, 16, 8), (2, 4, 10, 12)]:
        check(gb, w, Bu, Bv, ref=ref, bin_u=bu, bin_v=bv)


def test_lazy_empty_and_single(gb):
    G, S, O = 32, 7, 8
    plan = gb.Plan(G, S, O, 1, Bu=4, Bv=2, schedule="lazy")
    tab = torch.from_numpy(kb32(S, O).astype(np.float32)).cuda()
    g = torch.zeros((1, G, G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, torch.empty((0, 2), dtype=torch.float64, device="cuda"),
            torch.empty((0, 1), dtype=torch.complex64, device="cuda"), None, tab, g)
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0
    w = synth.Workload("one", G, S, O, 1, np.array([[1.25, -3.375]]), np.array([[2 - 1j]], np.complex64),
                       np.ones(1, np.float32))
    check(gb, w, 4, 2)
    check(gb, w, 8, 2, bin_u=24, bin_v=10)


@pytest.mark.parametrize("precision", ["bf16", "f16"])
def test_lazy_16bit_storage(gb, precision):
    """16-bit values and taps, FP32 accumulation: against the oracle on the same rounded inputs."""
    w = synth.scaled_down(quad_pol(), 60_000)
    dt = torch.bfloat16 if precision == "bf16" else torch.float16
    vis16 = torch.view_as_real(torch.from_numpy(w.vis)).to(dt)
    t16 = torch.from_numpy(kb32(w.S, w.oversample).astype(np.float32)).to(dt)
    vis_r = torch.view_as_complex(vis16.float().contiguous()).numpy().astype(np.complex128)
    tab_r = t16.float().numpy().astype(np.float64)
    ref, sk = oracle.grid(w.G, w.S, w.oversample, w.uv, vis_r, w.weights, tab_r)
    plan = gb.Plan(w.G, w.S, w.oversample, 4, Bu=4, Bv=2, schedule="lazy", precision=precision)
    g = torch.zeros((4, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, torch.from_numpy(w.uv).cuda(), vis16.cuda(), torch.from_numpy(w.weights).cuda(), t16.cuda(), g)
    got = g.cpu().numpy()
    assert plan.skipped() == sk
    for p in range(4):
        assert rel_l2(got[p], ref[p]) <= TOL


def test_lazy_plan_validation(gb):
    """Bins that are not multiples of the block, narrower than the paper's, or that make a team
    wider than a warp are refused at plan creation; so are unbuilt shapes and partial warps."""
    with pytest.raises(gb.GridderError) as e:
        gb.Plan(256, 7, 8, 4, Bu=4, Bv=2, schedule="lazy", bin_u=13, bin_v=10)
    assert e.value.code == -1
    with pytest.raises(gb.GridderError) as e:
        gb.Plan(256, 7, 8, 4, Bu=4, Bv=2, schedule="lazy", bin_u=8, bin_v=10)
    assert e.value.code == -1
    with pytest.raises(gb.GridderError) as e:
        gb.Plan(256, 7, 8, 4, Bu=2, Bv=2, schedule="lazy", bin_u=12, bin_v=12)
    assert e.value.code == -2
    with pytest.raises(gb.GridderError) as e:
        gb.Plan(256, 7, 8, 4, Bu=3, Bv=3, schedule="lazy")
    assert e.value.code == -2
    with pytest.raises(gb.GridderError) as e:
        gb.Plan(256, 7, 8, 4, Bu=4, Bv=2, schedule="lazy", threads=48)
    assert e.value.code == -1
    with pytest.raises(gb.GridderError) as e:
        gb.Plan(256, 7, 8, 4, Bu=2, Bv=2, schedule="chunked", bin_u=10)
    assert e.value.code == -1
    # default bins: one more block only where the paper's bin leaves less than a block of room
    for (Bu, Bv), want in {(4, 2): (12, 10, 15), (2, 2): (10, 10, 25), (2, 4): (10, 12, 15), (8, 1): (16, 8, 16),
                           (2, 1): (8, 8, 32)}.items():
        d = gb.Plan(256, 7, 8, 4, Bu=Bu, Bv=Bv, schedule="lazy").describe()
        assert (d["bin_u"], d["bin_v"], d["team_size"]) == want, (Bu, Bv, d)


def test_lazy_degrid_with_the_same_plan(gb):
    """degrid() with a lazy plan runs the chunked degridder on the paper's bin: oracle adjoint."""
    w = synth.scaled_down(quad_pol(), 50_000)
    table32 = kb32(w.S, w.oversample)
    rng = np.random.default_rng(4)
    g = (rng.standard_normal((4, w.G, w.G)) + 1j * rng.standard_normal((4, w.G, w.G))).astype(np.complex64)
    plan = gb.Plan(w.G, w.S, w.oversample, 4, Bu=4, Bv=2, schedule="lazy")
    tab = torch.from_numpy(table32.astype(np.float32)).cuda()
    out = gb.degrid(plan, torch.from_numpy(w.uv).cuda(), torch.from_numpy(g).cuda(), tab).cpu().numpy()
    ref, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, g, table32)
    for p in range(4):
        assert rel_l2(out[:, p], ref[:, p]) <= TOL


def test_lazy_degrid_fallback_shape(gb):
    """A lazy plan whose block shape has no chunked kernel (8x8 at P=1) degrids with 2x2 blocks."""
    w = synth.scaled_down(synth.precision_single_pol(), 20_000)
    table32 = kb32(w.S, w.oversample)
    rng = np.random.default_rng(6)
    g = (rng.standard_normal((1, w.G, w.G)) + 1j * rng.standard_normal((1, w.G, w.G))).astype(np.complex64)
    plan = gb.Plan(w.G, w.S, w.oversample, 1, Bu=8, Bv=8, schedule="lazy", bin_u=24, bin_v=24)
    tab = torch.from_numpy(table32.astype(np.float32)).cuda()
    out = gb.degrid(plan, torch.from_numpy(w.uv).cuda(), torch.from_numpy(g).cuda(), tab).cpu().numpy()
    ref, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, g, table32)
    assert rel_l2(out[:, 0], ref[:, 0]) <= TOL


def test_lazy_status_clear(gb):
    """Normal calls leave the status flags clear (no bulk copy timed out)."""
    w = synth.scaled_down(quad_pol(), 10_000)
    plan = check(gb, w, 4, 2)
    assert plan.status() == 0


def test_full_quad_pol_lazy(gb):
    """All 8,257,536 quad-pol visibilities with the lazy gridder in the configuration the bench
    tunes to (4x2 blocks, 12x10 bin, 512 visibilities per team, 128-thread CTAs)."""
    w = quad_pol()
    check(gb, w, 4, 2, bin_u=12, bin_v=10, vis_per_chunk=512, threads=128)
