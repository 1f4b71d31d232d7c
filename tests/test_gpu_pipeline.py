"""grid_degrid_host(): one grid + degrid pass from pinned host buffers with the copies overlapped.

The pipelined call must give the oracle's grid and degridded values (rel L2 <= 1e-5 per
polarization) for inputs that span several chunks with a ragged last chunk, with and without
weights. The grid is zeroed by the call, so a second call gives the same result. An empty call
zeroes the grid. Plans that disagree are rejected.
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
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def pinned(x):
    return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()


@pytest.mark.parametrize("dsched", ["chunked", "tile"])
@pytest.mark.parametrize("weighted", [True, False])
def test_pipelined_pass_matches_oracle(gb, weighted, dsched):
    w = synth.scaled_down(synth.quad_pol(), 300_007)
    rng = np.random.default_rng(21)
    wt = rng.uniform(0.2, 2.0, w.n_vis).astype(np.float32) if weighted else None
    t64 = oracle.kb_table(w.S, w.oversample, w.beta).astype(np.float32).astype(np.float64)
    table = torch.from_numpy(t64.astype(np.float32)).cuda()
    gplan = gb.Plan(w.G, w.S, w.oversample, w.npol, B=2, vis_per_chunk=128, threads=128)
    dplan = gb.Plan(w.G, w.S, w.oversample, w.npol, B=2, schedule=dsched)
    h_uv, h_vis = pinned(w.uv), pinned(w.vis)
    h_wt = None if wt is None else pinned(wt)
    h_out = torch.empty((w.n_vis, w.npol), dtype=torch.complex64).pin_memory()
    h_grid = torch.empty((w.npol, w.G, w.G), dtype=torch.complex64).pin_memory()
    g = torch.full((w.npol, w.G, w.G), 7.0, dtype=torch.complex64, device="cuda")  # the call zeroes it
    for _ in range(2):
        gb.grid_degrid_host(gplan, dplan, h_uv, h_vis, h_wt, table, g, h_out, h_grid, chunk=65_536)
        torch.cuda.synchronize()
        ref_g, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, wt, t64)
        for p in range(w.npol):
            assert rel_l2(h_grid.numpy()[p], ref_g[p]) <= TOL
        # degridding reads the device grid just gridded, so compare with the oracle's adjoint of it
        ref_v, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, h_grid.numpy().astype(np.complex128), t64)
        for p in range(w.npol):
            assert rel_l2(h_out.numpy()[:, p], ref_v[:, p]) <= TOL
        assert np.array_equal(h_grid.numpy(), g.cpu().numpy())


def test_pipelined_pass_empty_and_mismatch(gb):
    plan = gb.Plan(64, 7, 8, 1, B=2)
    table = gb.grid_make_kernel_table(7, 8, 2.34 * 7)
    g = torch.ones((1, 64, 64), dtype=torch.complex64, device="cuda")
    empty = torch.zeros((0, 2), dtype=torch.float64).pin_memory()
    gb.grid_degrid_host(plan, plan, empty, torch.zeros((0, 1), dtype=torch.complex64).pin_memory(), None, table, g,
                        torch.zeros((0, 1), dtype=torch.complex64).pin_memory(),
                        work=(torch.zeros((0, 2), dtype=torch.float64, device="cuda"),
                              torch.zeros((0, 1), dtype=torch.complex64, device="cuda"), None,
                              torch.zeros((0, 1), dtype=torch.complex64, device="cuda")))
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0
    other = gb.Plan(64, 9, 8, 1, B=2)
    w = synth.random_uniform(64, 7, 8, 1, 100, seed=3)
    with pytest.raises(gb.GridderError):
        gb.grid_degrid_host(plan, other, pinned(w.uv), pinned(w.vis), None, table, g,
                            torch.empty((100, 1), dtype=torch.complex64).pin_memory())


@pytest.mark.parametrize("dsched,chunk", [("chunked", 32_768), ("tile", 32_768), ("tile", 0)])
@pytest.mark.parametrize("weighted", [True, False])
def test_pipelined_steps_match_oracle(gb, weighted, dsched, chunk):
    base = synth.scaled_down(synth.quad_pol(), 120_001)
    rng = np.random.default_rng(22)
    t64 = oracle.kb_table(base.S, base.oversample, base.beta).astype(np.float32).astype(np.float64)
    table = torch.from_numpy(t64.astype(np.float32)).cuda()
    gplan = gb.Plan(base.G, base.S, base.oversample, base.npol, B=2, vis_per_chunk=128, threads=128)
    dplan = gb.Plan(base.G, base.S, base.oversample, base.npol, B=2, schedule=dsched, threads=32 if dsched == "tile" else 0)
    steps, want = [], []
    for s in range(3):
        # each step: the same tracks with its own values and weights
        vis = (rng.standard_normal((base.n_vis, base.npol)) + 1j * rng.standard_normal((base.n_vis, base.npol))).astype(np.complex64)
        wt = rng.uniform(0.2, 2.0, base.n_vis).astype(np.float32) if weighted else None
        steps.append(dict(uv=pinned(base.uv), vis=pinned(vis), weights=None if wt is None else pinned(wt),
                          vis_out=torch.empty((base.n_vis, base.npol), dtype=torch.complex64).pin_memory(),
                          grid_out=torch.empty((base.npol, base.G, base.G), dtype=torch.complex64).pin_memory()))
        want.append((vis, wt))
    g = torch.zeros((base.npol, base.G, base.G), dtype=torch.complex64, device="cuda")
    gb.grid_degrid_host_steps(gplan, dplan, steps, table, g, chunk=chunk)   # 0: the default chunk
    torch.cuda.synchronize()
    for st, (vis, wt) in zip(steps, want):
        ref_g, _ = oracle.grid(base.G, base.S, base.oversample, base.uv, vis, wt, t64)
        got_g = st["grid_out"].numpy()
        for p in range(base.npol):
            assert rel_l2(got_g[p], ref_g[p]) <= TOL
        ref_v, _ = oracle.degrid(base.G, base.S, base.oversample, base.uv, got_g.astype(np.complex128), t64)
        for p in range(base.npol):
            assert rel_l2(st["vis_out"].numpy()[:, p], ref_v[:, p]) <= TOL
