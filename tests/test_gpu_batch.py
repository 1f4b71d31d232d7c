"""Batched gridding (many grids, uneven counts, per-grid S) in one persistent launch, and in a CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_1605_07023_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1605_07023_gb300 as gb
    return gb


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def small_batch(n_chan=3, total=600_000, seed=0):
    """A reduced version of the batching workload: n_chan channels x 8 w-planes, G=1024, S by plane."""
    return synth.batched(seed=seed, n_chan=n_chan, total=total)


def device_items(ws):
    items = []
    for w in ws:
        t64 = oracle.kb_table(w.S, w.oversample, w.beta).astype(np.float32)
        items.append(dict(uv=torch.from_numpy(w.uv).cuda(), vis=torch.from_numpy(w.vis).cuda(),
                          weights=torch.from_numpy(w.weights).cuda(), table=torch.from_numpy(t64).cuda(),
                          grid=torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device="cuda"), S=w.S))
    return items


@pytest.mark.parametrize("B", [(2, 2), (1, 1), (3, 3), (4, 2)])
def test_batch_matches_oracle(gb, B):
    ws = [w for row in small_batch() for w in row]
    items = device_items(ws)
    bp = gb.BatchPlan(1024, 8, 1, Bu=B[0], Bv=B[1], max_S=15)
    bp.set(items)
    bp.execute()
    torch.cuda.synchronize()
    for w, it in zip(ws, items):
        ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, it["table"].cpu().numpy().astype(np.float64))
        assert rel_l2(it["grid"].cpu().numpy()[0], ref[0]) <= 1e-5, (w.name, B)
    assert bp.skipped() == 0


@pytest.mark.parametrize("shapes", [((2, 2), (4, 2), 13), ((2, 2), (4, 4), 11), ((2, 1), (2, 2), 9),
                                    ((2, 2), (2, 4), 11), ((1, 1), (3, 3), 10), ((4, 4), (2, 2), 9)])
def test_batch_two_shapes_matches_oracle(gb, shapes):
    (bu, bv), (bu2, bv2), split = shapes
    ws = [w for row in small_batch(n_chan=2, total=400_000, seed=4) for w in row]
    assert {w.S for w in ws} >= {7, 15} and any(w.S >= split for w in ws) and any(w.S < split for w in ws)
    items = device_items(ws)
    bp = gb.BatchPlan(1024, 8, 1, Bu=bu, Bv=bv, Bu2=bu2, Bv2=bv2, S_split=split, max_S=15)
    bp.set(items)
    bp.execute()
    torch.cuda.synchronize()
    for w, it in zip(ws, items):
        ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, it["table"].cpu().numpy().astype(np.float64))
        assert rel_l2(it["grid"].cpu().numpy()[0], ref[0]) <= 1e-5, (w.name, shapes)


@pytest.mark.parametrize("two", [False, True])
def test_batch_cuda_graph_replay(gb, two):
    """Replay of a captured batch: one launch, or one launch per block shape."""
    ws = [w for row in small_batch(n_chan=2, total=300_000, seed=1) for w in row]
    items = device_items(ws)
    shapes = dict(Bu2=4, Bv2=2, S_split=11) if two else {}
    bp = gb.BatchPlan(1024, 8, 1, Bu=2, Bv=2, max_S=15, **shapes)
    bp.set(items)
    bp.execute()                    # warm up outside the capture
    torch.cuda.synchronize()
    for it in items:
        it["grid"].zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bp.execute()
    for it in items:
        it["grid"].zero_()
    graph.replay()
    graph.replay()                  # gridding accumulates: two replays give twice the grid
    torch.cuda.synchronize()
    for w, it in zip(ws, items):
        ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, it["table"].cpu().numpy().astype(np.float64))
        assert rel_l2(it["grid"].cpu().numpy()[0], 2 * ref[0]) <= 1e-5


def test_batch_empty_and_invalid(gb):
    bp = gb.BatchPlan(64, 8, 1, Bu=2, Bv=2, max_S=7)
    bp.set([])
    bp.execute()
    w = synth.random_uniform(64, 7, 8, 1, 1000, seed=2)
    uv = w.uv.copy()
    uv[:10, 0] = 500.0                  # off the grid: skipped
    w.uv = uv
    items = device_items([w, synth.Workload("empty", 64, 7, 8, 1, np.zeros((0, 2)), np.zeros((0, 1), np.complex64),
                                            np.zeros(0, np.float32), beta=2.34 * 7)])
    bp.set(items)
    bp.execute()
    torch.cuda.synchronize()
    ref, sk = oracle.grid(64, 7, 8, w.uv, w.vis, w.weights, items[0]["table"].cpu().numpy().astype(np.float64))
    assert sk == 10 and bp.skipped() == 10
    assert rel_l2(items[0]["grid"].cpu().numpy()[0], ref[0]) <= 1e-5
    with pytest.raises(gb.GridderError):
        bad = dict(items[0], S=9)      # S above max_S
        bp.set([bad])


def test_batch_autotuner_picks_a_working_plan(gb):
    from paper_1605_07023_gb300 import autotune
    ws = [w for row in small_batch(n_chan=1, total=200_000, seed=5) for w in row]
    items = device_items(ws)
    best = autotune.tune_batch(1024, 8, 1, items, max_S=15, reps=1)
    assert best is not None and best["ms"] > 0
    cfg = {k: v for k, v in best.items() if k != "ms"}
    for it in items:
        it["grid"].zero_()
    bp = gb.BatchPlan(1024, 8, 1, max_S=15, **cfg)
    bp.set(items)
    bp.execute()
    torch.cuda.synchronize()
    for w, it in zip(ws, items):
        ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, it["table"].cpu().numpy().astype(np.float64))
        assert rel_l2(it["grid"].cpu().numpy()[0], ref[0]) <= 1e-5, (w.name, cfg)


def test_full_batching_workload(gb):
    """The whole batching workload (64 channels x 8 w-planes, 20 M visibilities, S by plane) in one
    launch with the tuned one-shape plan; every grid checked against the oracle."""
    ws = [w for row in synth.batched() for w in row]
    assert len(ws) == 512 and abs(sum(w.n_vis for w in ws) - 20_000_000) < 1000
    items = device_items(ws)
    bp = gb.BatchPlan(1024, 8, 1, Bu=2, Bv=2, max_S=15)
    bp.set(items)
    bp.execute()
    torch.cuda.synchronize()
    assert bp.skipped() == 0
    for w, it in zip(ws, items):
        ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, it["table"].cpu().numpy().astype(np.float64))
        assert rel_l2(it["grid"].cpu().numpy()[0], ref[0]) <= 1e-5, w.name


def test_batch_two_shapes_quad_pol(gb):
    """Four polarizations, two shapes (2x1 below S=9, 2x2 above)."""
    rng = np.random.default_rng(8)
    ws = []
    for k, S in enumerate((7, 7, 9, 11)):
        w = synth.scaled_down(synth.quad_pol(seed=k), 20_000 + 777 * k)
        ws.append(synth.Workload(f"qp{k}", w.G, S, w.oversample, 4, w.uv * 0.9, w.vis, rng.uniform(0.5, 2, w.n_vis).astype(np.float32),
                                 beta=2.34 * S))
    items = device_items(ws)
    bp = gb.BatchPlan(2048, 8, 4, Bu=2, Bv=1, Bu2=2, Bv2=2, S_split=9, max_S=11)
    bp.set(items)
    bp.execute()
    torch.cuda.synchronize()
    for w, it in zip(ws, items):
        ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, it["table"].cpu().numpy().astype(np.float64))
        got = it["grid"].cpu().numpy()
        for p in range(4):
            assert rel_l2(got[p], ref[p]) <= 1e-5, (w.name, p)
