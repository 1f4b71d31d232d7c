"""16-bit storage of visibilities and taps (bf16 / fp16), FP32 accumulation.

Two measures for each storage format:
  - parity (gated, rel L2 <= 1e-5): the CUDA path against the FP64 oracle fed
    the SAME 16-bit-rounded visibilities and taps, upcast exactly. This checks
    the kernels;
  - storage error (reported, loosely bounded): the same grid against the
    oracle on the unrounded FP32 inputs. This is the price of the format:
    about 2^-9 relative for bf16 and 2^-12 for fp16 per value, averaged down
    over many contributions.
"""
import functools

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


@functools.lru_cache(maxsize=None)
def precision_workload():
    return synth.precision_single_pol()


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def host_table(w, prec):
    """The oracle's FP64 table, rounded to the storage format on the host (the same input for both sides)."""
    tdt = torch.bfloat16 if prec == "bf16" else torch.float16
    return torch.from_numpy(oracle.kb_table(w.S, w.oversample, w.beta)).to(tdt).cuda()


def run(gb, w, prec, B, schedule="chunked"):
    tdt = torch.bfloat16 if prec == "bf16" else torch.float16
    vis16 = torch.view_as_real(torch.from_numpy(w.vis)).to(tdt).contiguous()          # [n, P, 2]
    table16 = host_table(w, prec)
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, B=B, precision=prec, schedule=schedule)
    g = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, torch.from_numpy(w.uv).cuda(), vis16.cuda(), torch.from_numpy(w.weights).cuda(), table16, g)
    torch.cuda.synchronize()
    vis_r = vis16.float().numpy()
    vis_r = (vis_r[..., 0] + 1j * vis_r[..., 1]).astype(np.complex128)
    return g.cpu().numpy(), vis_r, table16.float().cpu().numpy().astype(np.float64), plan


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("B,schedule", [(1, "chunked"), (2, "chunked"), (4, "chunked"), (2, "patch")])
def test_precision_subset(gb, prec, B, schedule):
    w = synth.scaled_down(precision_workload(), 400_000)
    got, vis_r, tab_r, plan = run(gb, w, prec, B, schedule)
    ref, sk = oracle.grid(w.G, w.S, w.oversample, w.uv, vis_r, w.weights, tab_r)
    assert plan.skipped() == sk
    assert rel_l2(got[0], ref[0]) <= 1e-5


@pytest.mark.parametrize("prec,bound", [("bf16", 2.0 ** -7), ("f16", 2.0 ** -10)])
def test_precision_full_workload(gb, prec, bound):
    """All 16,711,680 visibilities (G=4096, S=15, O=16): parity gated, storage error reported."""
    w = precision_workload()
    got, vis_r, tab_r, _ = run(gb, w, prec, 2)
    ref_same, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, vis_r, w.weights, tab_r)
    assert rel_l2(got[0], ref_same[0]) <= 1e-5
    t64 = oracle.kb_table(w.S, w.oversample, w.beta)
    ref_fp, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, t64)
    err = rel_l2(got[0], ref_fp[0])
    print(f"{prec}: rel L2 vs FP64 oracle on unrounded inputs = {err:.3e}")
    assert err <= bound


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_degrid_with_16bit_taps(gb, prec):
    w = synth.scaled_down(precision_workload(), 200_000)
    table16 = host_table(w, prec)
    tab_r = table16.float().cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(4)
    g = (rng.standard_normal((1, w.G, w.G)) + 1j * rng.standard_normal((1, w.G, w.G))).astype(np.complex64)
    plan = gb.Plan(w.G, w.S, w.oversample, 1, B=2, precision=prec)
    out = gb.degrid(plan, torch.from_numpy(w.uv).cuda(), torch.from_numpy(g).cuda(), table16)
    torch.cuda.synchronize()
    ref, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, g, tab_r)
    assert rel_l2(out.cpu().numpy()[:, 0], ref[:, 0]) <= 1e-5


@pytest.mark.parametrize("prec", ["bf16", "f16"])
@pytest.mark.parametrize("npol,B", [(2, 2), (4, 2), (4, 1), (2, 3)])
def test_precision_multi_polarization_weighted(gb, prec, npol, B):
    """16-bit values of 2 and 4 polarizations (one 64- or 128-bit load per record), non-unit weights,
    a ragged last chunk: FP32 accumulation against the oracle given the same rounded inputs."""
    base = synth.scaled_down(synth.quad_pol(), 50_001)
    rng = np.random.default_rng(40 + npol)
    wts = rng.uniform(0.1, 3.0, base.n_vis).astype(np.float32)
    vis = base.vis[:, :npol].copy()
    tdt = torch.bfloat16 if prec == "bf16" else torch.float16
    vis16 = torch.view_as_real(torch.from_numpy(vis)).to(tdt).contiguous()
    table16 = host_table(base, prec)
    plan = gb.Plan(base.G, base.S, base.oversample, npol, B=B, precision=prec)
    g = torch.zeros((npol, base.G, base.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, torch.from_numpy(base.uv).cuda(), vis16.cuda(), torch.from_numpy(wts).cuda(), table16, g)
    torch.cuda.synchronize()
    vis_r = vis16.float().numpy()
    vis_r = (vis_r[..., 0] + 1j * vis_r[..., 1]).astype(np.complex128)
    ref, sk = oracle.grid(base.G, base.S, base.oversample, base.uv, vis_r, wts,
                          table16.float().cpu().numpy().astype(np.float64))
    assert plan.skipped() == sk
    got = g.cpu().numpy()
    for p in range(npol):
        assert rel_l2(got[p], ref[p]) <= 1e-5, p
