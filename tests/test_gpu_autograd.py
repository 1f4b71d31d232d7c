"""Differentiation through the CUDA gridder: backward = the degridding kernel.

Checks:
  - GridFn's backward equals the oracle's weighted adjoint, w * degrid(grad);
  - DegridFn's backward equals the oracle's grid() of the incoming gradient;
  - the differentiation workload: loss = ||FFT(grid(vis)) - target||^2 with a
    seeded Gaussian-source target image. The analytic gradient on 32 random
    visibilities (real and imaginary parts) matches central finite
    differences to 1e-3 relative.

The loss is quadratic in vis, so central differences are exact up to rounding.
They are formed as g0 +- h * grid(e_k), where grid(e_k) is the GPU kernel's
own gridding of one unit visibility. The finite difference then measures the
forward kernel, not the FP32 summation-order noise of regridding a million
visibilities.
"""
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


def kb32(w):
    """The oracle's KB table rounded to FP32 on the host, as float64 (the same input for both sides)."""
    return oracle.kb_table(w.S, w.oversample, w.beta).astype(np.float32).astype(np.float64)


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("schedule", ["chunked", "patch", "tile"])
def test_grid_backward_is_weighted_adjoint(gb, schedule):
    from paper_1605_07023_gb300.autograd import grid_op
    w = synth.scaled_down(synth.quad_pol(), 60_000)
    rng = np.random.default_rng(1)
    wt = rng.uniform(0.2, 2.0, w.n_vis).astype(np.float32)
    t64 = kb32(w)
    table = torch.from_numpy(t64.astype(np.float32)).cuda()
    plan = gb.Plan(w.G, w.S, w.oversample, 4, B=2, schedule=schedule)
    uv = torch.from_numpy(w.uv).cuda()
    vis = torch.from_numpy(w.vis).cuda().requires_grad_(True)
    wtt = torch.from_numpy(wt).cuda()
    g = grid_op(plan, uv, vis, wtt, table)
    gg = (rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)).astype(np.complex64)
    g.backward(torch.from_numpy(gg).cuda())
    ref, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, gg, t64)
    ref = ref * wt[:, None]
    got = vis.grad.cpu().numpy()
    for p in range(4):
        assert rel_l2(got[:, p], ref[:, p]) <= 1e-5


def test_degrid_backward_is_grid(gb):
    from paper_1605_07023_gb300.autograd import degrid_op
    w = synth.scaled_down(synth.quad_pol(), 40_000)
    t64 = kb32(w)
    table = torch.from_numpy(t64.astype(np.float32)).cuda()
    plan = gb.Plan(w.G, w.S, w.oversample, 4, B=2)
    rng = np.random.default_rng(2)
    g0 = (rng.standard_normal((4, w.G, w.G)) + 1j * rng.standard_normal((4, w.G, w.G))).astype(np.complex64)
    gt = torch.from_numpy(g0).cuda().requires_grad_(True)
    v = degrid_op(plan, torch.from_numpy(w.uv).cuda(), gt, table)
    gv = (rng.standard_normal(v.shape) + 1j * rng.standard_normal(v.shape)).astype(np.complex64)
    v.backward(torch.from_numpy(gv).cuda())
    ref, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, gv, None, t64)
    got = gt.grad.cpu().numpy()
    for p in range(4):
        assert rel_l2(got[p], ref[p]) <= 1e-5


def test_differentiation_workload_finite_differences(gb):
    from paper_1605_07023_gb300.autograd import grid_op
    w = synth.differentiation()
    assert w.n_vis == 1_000_000
    target = torch.from_numpy(synth.gaussian_sources_image(w.G, 5, seed=0)).cuda()
    table = torch.from_numpy(kb32(w).astype(np.float32)).cuda()
    plan = gb.Plan(w.G, w.S, w.oversample, 1, B=2)
    uv = torch.from_numpy(w.uv).cuda()
    wt = torch.from_numpy(w.weights).cuda()

    def image(g):  # FFT of the FP32 grid, in FP64
        return torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(g.to(torch.complex128)[0]), norm="forward"))

    def loss_of_grid(g):  # loss = sum |FFT(grid) - target|^2
        return torch.sum(torch.abs(image(g) - target) ** 2)

    vis = torch.from_numpy(w.vis).cuda().requires_grad_(True)
    g = grid_op(plan, uv, vis, wt, table)
    loss = loss_of_grid(g)
    loss.backward()
    grad = vis.grad.detach().cpu().numpy()[:, 0]
    g0 = g.detach()

    rng = np.random.default_rng(3)
    ks = rng.choice(w.n_vis, 32, replace=False)
    h = 1e-2 * float(np.sqrt(np.mean(np.abs(w.vis) ** 2)))
    worst = 0.0
    for k in ks:
        one = torch.zeros((1, 1), dtype=torch.complex64, device="cuda")
        gk = torch.zeros_like(g0)
        fd = {}
        for part, dv in (("re", 1.0 + 0j), ("im", 1j)):
            one.fill_(dv)
            gk.zero_()
            gb.grid(plan, uv[k:k + 1].contiguous(), one, wt[k:k + 1].contiguous(), table, gk)
            # central difference L(g0 + h gk) - L(g0 - h gk), differenced pixel by pixel before the
            # sum: the loss is about 1e16 and the difference about 1e2, so subtracting the two sums
            # would lose the difference to FP64 rounding
            rp = torch.abs(image(g0 + h * gk) - target) ** 2
            rm = torch.abs(image(g0 - h * gk) - target) ** 2
            fd[part] = float(torch.sum(rp - rm)) / (2 * h)
        # PyTorch's complex gradient is dL/dRe + i dL/dIm; compare as complex numbers, relative to
        # the gradient's magnitude at this visibility (one component can be 1000x the other)
        fdc = fd["re"] + 1j * fd["im"]
        err = abs(fdc - grad[k]) / abs(grad[k])
        worst = max(worst, err)
        assert err <= 1e-3, (k, fdc, grad[k])
    assert worst <= 1e-3

    # the whole gradient against an FP64 pipeline built from the oracle: oracle grid, FP64 FFT,
    # oracle adjoint (degrid) of dL/dgrid
    t64 = kb32(w)
    g64, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, w.vis, w.weights, t64)
    tgt = synth.gaussian_sources_image(w.G, 5, seed=0)
    A = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(g64[0]), norm="forward")) - tgt
    dLdg = 2 * np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(A), norm="backward"))  # adjoint of the unnormalised inverse FFT
    ref, _ = oracle.degrid(w.G, w.S, w.oversample, w.uv, dLdg[None], t64)
    ref = ref[:, 0] * w.weights
    assert np.linalg.norm(grad - ref) / np.linalg.norm(ref) <= 1e-5
