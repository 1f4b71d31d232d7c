"""Compression (grid_compress) and expansion (degrid_expand) on the GPU against the oracle.

Compression is index work decided by the exact fine-position rule, so the run
assignment (run_of), the run count and the copied uv of each run are compared
bit for bit. The merged values are FP32 sums of w*V in input order and are
compared per polarization by relative L2 against the oracle's FP64 sums.
Gridding the merged records, and degridding them then expanding, must give the
oracle's results on the original records (Sec. 2.2: compression leaves the
grid unchanged up to rounding).
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def compress_both(gb, plan, O, uv, vis, weights):
    uv_c, vis_c, run_of = gb.grid_compress(plan, dev(uv), dev(vis), None if weights is None else dev(weights))
    ouv, ovis, orun = oracle.compress(O, uv, vis, weights)
    return (uv_c.cpu().numpy(), vis_c.cpu().numpy(), run_of.cpu().numpy()), (ouv, ovis, orun)


def assert_same(got, want):
    (uv_c, vis_c, run_of), (ouv, ovis, orun) = got, want
    assert len(uv_c) == len(ouv)
    assert np.array_equal(run_of, orun)
    assert np.array_equal(uv_c, ouv, equal_nan=True)
    for p in range(ovis.shape[1]):
        assert rel_l2(vis_c[:, p], ovis[:, p]) <= TOL, p


@pytest.mark.parametrize("case", ["plain", "cored300k"])
def test_compress_matches_oracle(gb, case):
    w = synth.plain_single_pol() if case == "plain" else synth.scaled_down(synth.cored_quad_pol(), 300_007)
    rng = np.random.default_rng(11)
    wt = rng.uniform(0.2, 2.0, w.n_vis).astype(np.float32)
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, B=2)
    got, want = compress_both(gb, plan, w.oversample, w.uv, w.vis, wt)
    assert len(want[0]) < w.n_vis
    assert_same(got, want)


def test_compress_full_cored_workload(gb):
    w = synth.cored_quad_pol()
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, B=2)
    got, want = compress_both(gb, plan, w.oversample, w.uv, w.vis, w.weights)
    assert 0.5 * w.n_vis < len(want[0]) < 0.6 * w.n_vis
    assert_same(got, want)


def test_compressed_grid_and_degrid_match_oracle_on_originals(gb):
    w = synth.scaled_down(synth.cored_quad_pol(), 200_000)
    rng = np.random.default_rng(12)
    wt = rng.uniform(0.2, 2.0, w.n_vis).astype(np.float32)
    t64 = oracle.kb_table(w.S, w.oversample, w.beta).astype(np.float32).astype(np.float64)
    table = dev(t64.astype(np.float32))
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, B=2)
    uv_c, vis_c, run_of = gb.grid_compress(plan, dev(w.uv), dev(w.vis), dev(wt))
    assert uv_c.shape[0] < 0.7 * w.n_vis
    g = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, uv_c, vis_c, None, table, g)
    ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, wt, t64)
    got = g.cpu().numpy()
    for p in range(w.npol):
        assert rel_l2(got[p], ref[p]) <= TOL
    # degrid the merged records, expand to the originals (with and without weights)
    gr = (rng.standard_normal((w.npol, w.G, w.G)) + 1j * rng.standard_normal((w.npol, w.G, w.G))).astype(np.complex64)
    dc = gb.degrid(plan, uv_c, dev(gr), table)
    d = gb.degrid_expand(plan, run_of, dc).cpu().numpy()
    dw = gb.degrid_expand(plan, run_of, dc, dev(wt)).cpu().numpy()
    dref, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, gr.astype(np.complex128), t64)
    for p in range(w.npol):
        assert rel_l2(d[:, p], dref[:, p]) <= TOL
        assert rel_l2(dw[:, p], wt * dref[:, p]) <= TOL


def test_compress_16bit_inputs(gb):
    w = synth.scaled_down(synth.cored_quad_pol(), 100_000)
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, B=2, precision="bf16")
    v16 = torch.from_numpy(w.vis.view(np.float32)).to(torch.bfloat16)          # [n, 2P] interleaved
    v_round = v16.to(torch.float32).numpy().view(np.complex64)                  # what the kernel reads, exactly
    uv_c, vis_c, run_of = gb.grid_compress(plan, dev(w.uv), v16.reshape(w.n_vis, 2 * w.npol).cuda(), dev(w.weights))
    want = oracle.compress(w.oversample, w.uv, v_round, w.weights)
    assert_same((uv_c.cpu().numpy(), vis_c.cpu().numpy(), run_of.cpu().numpy()), want)


def test_compress_edge_cases(gb):
    O = 8
    plan = gb.Plan(64, 7, O, 1, B=2)
    # empty and single
    for n in (0, 1):
        uv = np.full((n, 2), 3.0)
        vis = np.ones((n, 1), np.complex64)
        got, want = compress_both(gb, plan, O, uv, vis, None)
        assert_same(got, want)
    # a stationary run across five tiles of 1024, then alternation, NaN and far-off coordinates
    rng = np.random.default_rng(13)
    uv = np.concatenate([np.full((5000, 2), 3.0) + rng.uniform(-0.3, 0.3, (5000, 2)) / O,
                         np.tile([[3.0, 4.0], [5.0, 4.0]], (700, 1)),
                         [[np.nan, 1.0], [np.nan, 1.0], [1.0, np.inf], [1e9, 1.0], [1e9, 1.0], [2.0**23 / O, 0.0],
                          [2.0**23 / O, 0.0], [1.0, 1.0], [1.0, 1.0]]])
    n = len(uv)
    vis = (rng.standard_normal((n, 1)) + 1j * rng.standard_normal((n, 1))).astype(np.complex64)
    got, want = compress_both(gb, plan, O, uv, vis, rng.uniform(0.5, 1.5, n).astype(np.float32))
    assert want[2][4999] == 0 and len(want[0]) == 1 + 1400 + 7
    assert_same(got, want)


def test_expand_out_of_range_run_gives_zero(gb):
    plan = gb.Plan(64, 7, 8, 2, B=2)
    run_of = torch.tensor([0, 1, -1, 2, 7], dtype=torch.int64, device="cuda")
    vc = torch.arange(6, dtype=torch.float32, device="cuda").reshape(3, 2).to(torch.complex64)
    out = gb.degrid_expand(plan, run_of, vc).cpu().numpy()
    want = np.array([[0, 1], [2, 3], [0, 0], [4, 5], [0, 0]], np.complex64)
    assert np.array_equal(out, want)
