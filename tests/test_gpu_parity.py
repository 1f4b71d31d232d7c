"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bars:
  - cell indices and table rows: bit-exact;
  - grid and degrid values: relative L2 error <= 1e-5 per polarization plane
    (FP32 accumulation against FP64).
Every case runs on the same seeded inputs on both sides.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1605_07023_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@functools.lru_cache(maxsize=None)
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
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def to_dev(w, table64, precision="f32"):
    uv = torch.from_numpy(np.ascontiguousarray(w.uv)).cuda()
    vis = torch.from_numpy(np.ascontiguousarray(w.vis)).cuda()
    wt = torch.from_numpy(np.ascontiguousarray(w.weights)).cuda()
    tab = torch.from_numpy(table64.astype(np.float32)).cuda()
    return uv, vis, wt, tab


def kb32(S, O):
    return oracle.kb_table(S, O, 2.34 * S).astype(np.float32).astype(np.float64)


def run_grid(gb, w, plan, table32):
    uv, vis, wt, tab = to_dev(w, table32)
    g = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, uv, vis, wt, tab, g)
    torch.cuda.synchronize()
    return g.cpu().numpy()


def check_grid(gb, w, Bu, Bv, schedule="chunked", **kw):
    table32 = kb32(w.S, w.oversample)
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, Bu=Bu, Bv=Bv, schedule=schedule, **kw)
    got = run_grid(gb, w, plan, table32)
    ref, sk = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, table32)
    assert plan.skipped() == sk
    for p in range(w.npol):
        e = rel_l2(got[p], ref[p])
        assert e <= TOL, (Bu, Bv, schedule, p, e)
    return plan


# ------------------------------------------------------------------ indices

def test_indices_bit_exact(gb):
    w = synth.plain_single_pol()
    O = w.oversample
    rng = np.random.default_rng(11)
    ties = (rng.integers(-1000, 1000, 4000) + 0.5) / O
    edge = np.concatenate([ties, np.nextafter(ties, np.inf), np.nextafter(ties, -np.inf),
                           [np.nan, np.inf, -np.inf, 1e300, -1e300, 0.0, -0.0, 5e-324, -5e-324, 127.0, -128.0, 124.0, -125.0]])
    uv = np.concatenate([w.uv, np.stack([edge, rng.permutation(edge)], 1), rng.uniform(-140, 140, (5000, 2))])
    plan = gb.Plan(w.G, w.S, O, 1)
    cell, sub = gb.grid_compute_indices(plan, torch.from_numpy(uv).cuda())
    rc, rs, _ = oracle.indices(w.G, w.S, O, uv)
    np.testing.assert_array_equal(cell.cpu().numpy(), rc)
    np.testing.assert_array_equal(sub.cpu().numpy(), rs)


@pytest.mark.parametrize("S,O", [(7, 8), (15, 16), (1, 1), (9, 64)])
def test_indices_bit_exact_other_geometries(gb, S, O):
    G = 512
    rng = np.random.default_rng(S * 100 + O)
    f = rng.integers(-G * O // 2, G * O // 2, (20000, 2))
    uv = np.concatenate([f / O, (f + 0.5) / O, rng.uniform(-G / 2, G / 2, (20000, 2))])
    plan = gb.Plan(G, S, O, 1)
    cell, sub = gb.grid_compute_indices(plan, torch.from_numpy(uv).cuda())
    rc, rs, _ = oracle.indices(G, S, O, uv)
    np.testing.assert_array_equal(cell.cpu().numpy(), rc)
    np.testing.assert_array_equal(sub.cpu().numpy(), rs)


# ------------------------------------------------------------------ kernel table

@pytest.mark.parametrize("S,O", [(7, 8), (15, 16), (9, 8), (11, 8)])
def test_kernel_table_matches_oracle(gb, S, O):
    beta = 2.34 * S
    t = gb.grid_make_kernel_table(S, O, beta).cpu().numpy().astype(np.float64)
    ref = oracle.kb_table(S, O, beta)
    # both are FP64 evaluations (different I0 algorithms) rounded once to FP32
    np.testing.assert_allclose(t, ref, rtol=1.2e-7, atol=0)
    for prec, eps in (("bf16", 2.0 ** -8), ("f16", 2.0 ** -11)):
        t16 = gb.grid_make_kernel_table(S, O, beta, prec).float().cpu().numpy()
        np.testing.assert_allclose(t16, ref, rtol=eps * 1.01, atol=6e-8)


# ------------------------------------------------------------------ gridding parity

BLOCKS = [(1, 1), (2, 1), (1, 2), (2, 2), (3, 3), (4, 2), (2, 4), (4, 4), (8, 1), (1, 8), (8, 2), (2, 8), (4, 1), (1, 4)]


@pytest.mark.parametrize("Bu,Bv", BLOCKS)
def test_grid_plain_single_pol(gb, Bu, Bv):
    """The 30,720-visibility G=256 single-pol workload, every coarsening shape."""
    check_grid(gb, synth.plain_single_pol(), Bu, Bv)


@pytest.mark.parametrize("Bu,Bv", [(1, 1), (2, 2), (2, 1), (4, 2), (3, 3), (4, 4)])
@pytest.mark.parametrize("schedule", ["chunked", "patch"])
def test_grid_quad_pol_subset(gb, Bu, Bv, schedule):
    """The first 200,001 visibilities of the quad-pol G=2048 workload (a ragged tail)."""
    w = synth.scaled_down(quad_pol(), 200_001)
    check_grid(gb, w, Bu, Bv, schedule)


@pytest.mark.parametrize("schedule", ["chunked", "patch"])
@pytest.mark.parametrize("npol", [1, 2, 4])
def test_grid_random_positions_and_weights(gb, schedule, npol):
    """Unordered positions (no coherence), non-unit weights, every P."""
    w = synth.random_uniform(300, 9, 8, npol, 50_003, seed=npol)
    w.weights = np.random.default_rng(3).uniform(0.1, 2.0, w.n_vis).astype(np.float32)
    check_grid(gb, w, 2, 2, schedule)
    check_grid(gb, w, 1, 1, schedule)


@pytest.mark.parametrize("npol", [1, 4])
@pytest.mark.parametrize("Bu,Bv", [(1, 1), (2, 1), (3, 3), (4, 4), (2, 2)])
@pytest.mark.parametrize("threads", [0, 224, 1000])
def test_patch_schedule_partial_warps(gb, npol, Bu, Bv, threads):
    """Patch schedule for team sizes that leave a partial last warp (49, 28, 9 threads per team)."""
    w = synth.random_uniform(256, 7, 8, npol, 30_011, seed=Bu * 10 + Bv + npol)
    try:
        check_grid(gb, w, Bu, Bv, "patch", threads=threads)
    except gb.GridderError as e:      # a CTA size that cannot hold the window is refused, not run
        assert e.code == -2


@pytest.mark.parametrize("chunk", [1, 7, 16, 33, 1024])
def test_grid_chunk_lengths(gb, chunk):
    w = synth.scaled_down(quad_pol(), 40_000)
    check_grid(gb, w, 2, 2, vis_per_chunk=chunk)
    check_grid(gb, w, 2, 2, "patch", vis_per_chunk=chunk)


def test_grid_large_support(gb):
    """S=15, O=16 (the precision workload's kernel) on a subset, plain and coarsened."""
    w = synth.scaled_down(synth.precision_single_pol(), 100_000)
    for B in [(1, 1), (2, 2), (4, 4), (3, 3)]:
        check_grid(gb, w, *B)
    check_grid(gb, w, 2, 2, "patch")


def test_grid_edges_and_invalid(gb):
    """Footprints touching every grid edge, plus invalid and off-grid visibilities."""
    G, S, O = 64, 7, 8
    h = 3
    lo, hi = h - G // 2, G // 2 - h - 1
    rng = np.random.default_rng(5)
    pts = [[lo, lo], [hi, hi], [lo, hi], [hi, lo], [lo - 0.5, 0], [hi + 0.49, 0.2], [0, hi + 0.5], [np.nan, 0],
           [0, np.inf], [1e9, 0], [-40, 0]]
    uv = np.concatenate([np.array(pts, float), rng.uniform(lo - 2, hi + 2, (3000, 2))])
    vis = (rng.standard_normal((len(uv), 4)) + 1j * rng.standard_normal((len(uv), 4))).astype(np.complex64)
    w = synth.Workload("edges", G, S, O, 4, uv, vis, np.ones(len(uv), np.float32))
    for B in [(1, 1), (2, 2), (3, 3), (8, 2)]:
        for sched in ("chunked", "patch"):
            check_grid(gb, w, *B, sched)


def test_grid_empty_and_single(gb):
    G, S, O = 32, 7, 8
    plan = gb.Plan(G, S, O, 1, B=2)
    tab = torch.from_numpy(kb32(S, O).astype(np.float32)).cuda()
    g = torch.zeros((1, G, G), dtype=torch.complex64, device="cuda")
    e = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    gb.grid(plan, e, torch.empty((0, 1), dtype=torch.complex64, device="cuda"), None, tab, g)
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0
    w = synth.Workload("one", G, S, O, 1, np.array([[1.25, -3.375]]), np.array([[2 - 1j]], np.complex64),
                       np.ones(1, np.float32))
    check_grid(gb, w, 2, 2)
    check_grid(gb, w, 1, 1, "patch")


def test_plans_sharing_a_kernel_do_not_interfere(gb):
    """A patch plan still launches after a chunked plan with the same (Bu, Bv, P) was created."""
    w = synth.scaled_down(quad_pol(), 30_000)
    table32 = kb32(w.S, w.oversample)
    p_patch = gb.Plan(w.G, w.S, w.oversample, 4, B=2, schedule="patch")
    p_chunk = gb.Plan(w.G, w.S, w.oversample, 4, B=2, schedule="chunked")
    ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, table32)
    for plan in (p_patch, p_chunk, p_patch):
        got = run_grid(gb, w, plan, table32)
        assert max(rel_l2(got[p], ref[p]) for p in range(4)) <= TOL


def test_grid_accumulates(gb):
    """grid() adds to what is already in the grid."""
    w = synth.plain_single_pol()
    table32 = kb32(w.S, w.oversample)
    plan = gb.Plan(w.G, w.S, w.oversample, 1, B=2)
    uv, vis, wt, tab = to_dev(w, table32)
    g = torch.zeros((1, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, uv, vis, wt, tab, g)
    gb.grid(plan, uv, vis, wt, tab, g)
    ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, table32)
    assert rel_l2(g.cpu().numpy()[0], 2 * ref[0]) <= TOL


# ------------------------------------------------------------------ degridding parity

def check_degrid(gb, w, Bu, Bv, seed=0):
    table32 = kb32(w.S, w.oversample)
    rng = np.random.default_rng(seed)
    g64 = (rng.standard_normal((w.npol, w.G, w.G)) + 1j * rng.standard_normal((w.npol, w.G, w.G))).astype(np.complex64)
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, Bu=Bu, Bv=Bv)
    uv = torch.from_numpy(np.ascontiguousarray(w.uv)).cuda()
    tab = torch.from_numpy(table32.astype(np.float32)).cuda()
    out = gb.degrid(plan, uv, torch.from_numpy(g64).cuda(), tab)
    torch.cuda.synchronize()
    ref, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, g64, table32)
    got = out.cpu().numpy()
    for p in range(w.npol):
        e = rel_l2(got[:, p], ref[:, p])
        assert e <= TOL, (Bu, Bv, p, e)


@pytest.mark.parametrize("Bu,Bv", BLOCKS)
def test_degrid_plain_single_pol(gb, Bu, Bv):
    check_degrid(gb, synth.plain_single_pol(), Bu, Bv)


@pytest.mark.parametrize("Bu,Bv", [(1, 1), (2, 2), (4, 2), (3, 3)])
def test_degrid_quad_pol_subset(gb, Bu, Bv):
    check_degrid(gb, synth.scaled_down(quad_pol(), 100_003), Bu, Bv)


def test_degrid_edges_random(gb):
    w = synth.random_uniform(64, 7, 8, 2, 20_001, seed=9)
    for B in [(1, 1), (2, 2), (8, 1)]:
        check_degrid(gb, w, *B)


def test_adjoint_on_gpu(gb):
    """<grid(v), g> = <v, degrid(g)> for the CUDA pair, to FP32 accuracy."""
    w = synth.scaled_down(quad_pol(), 50_000)
    table32 = kb32(w.S, w.oversample)
    rng = np.random.default_rng(12)
    g = (rng.standard_normal((4, w.G, w.G)) + 1j * rng.standard_normal((4, w.G, w.G))).astype(np.complex64)
    plan = gb.Plan(w.G, w.S, w.oversample, 4, B=2)
    uv, vis, _, tab = to_dev(w, table32)
    gv = torch.zeros((4, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, uv, vis, None, tab, gv)
    dg = gb.degrid(plan, uv, torch.from_numpy(g).cuda(), tab)
    lhs = np.vdot(gv.cpu().numpy().astype(np.complex128), g.astype(np.complex128))
    rhs = np.vdot(w.vis.astype(np.complex128), dg.cpu().numpy().astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


# ------------------------------------------------------------------ full-size quad-pol workload

@pytest.mark.parametrize("schedule,B", [("chunked", (1, 1)), ("chunked", (2, 2)), ("patch", (2, 2))])
def test_full_quad_pol(gb, schedule, B):
    """All 8,257,536 visibilities, in the launch configurations the benchmark times."""
    w = quad_pol()
    check_grid(gb, w, *B, schedule)


def test_full_quad_pol_bench_launch_configs(gb):
    """All 8,257,536 visibilities in the configurations the bench tunes to and times: gridding with
    2x2 blocks, 128 visibilities per team and 128-thread CTAs, the plain Romein kernel (B=1, 1024 per
    team), and degridding with 2x2 blocks, 64 per team and 256-thread CTAs (checked against the
    oracle's adjoint of the GPU grid)."""
    w = quad_pol()
    check_grid(gb, w, 2, 2, "chunked", vis_per_chunk=128, threads=128)
    check_grid(gb, w, 1, 1, "chunked", vis_per_chunk=1024)
    table32 = kb32(w.S, w.oversample)
    gplan = gb.Plan(w.G, w.S, w.oversample, w.npol, Bu=2, Bv=2, vis_per_chunk=128, threads=128)
    got_grid = run_grid(gb, w, gplan, table32)
    dplan = gb.Plan(w.G, w.S, w.oversample, w.npol, Bu=2, Bv=2, vis_per_chunk=64, threads=256)
    uv, _, _, tab = to_dev(w, table32)
    dv = gb.degrid(dplan, uv, torch.from_numpy(got_grid.astype(np.complex64)).cuda(), tab).cpu().numpy()
    ref, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, got_grid.astype(np.complex64).astype(np.complex128), table32)
    for p in range(w.npol):
        assert rel_l2(dv[:, p], ref[:, p]) <= TOL
