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


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("schedule", ["chunked", "patch"])
def test_grid_backward_is_weighted_adjoint(gb, schedule):
    from paper_1605_07023_gb300.autograd import grid_op
    w = synth.scaled_down(synth.quad_pol(), 60_000)
    rng = np.random.default_rng(1)
    wt = rng.uniform(0.2, 2.0, w.n_vis).astype(np.float32)
    table = gb.grid_make_kernel_table(w.S, w.oversample, w.beta)
    t64 = table.cpu().numpy().astype(np.float64)
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
    table = gb.grid_make_kernel_table(w.S, w.oversample, w.beta)
    t64 = table.cpu().numpy().astype(np.float64)
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
    table = gb.grid_make_kernel_table(w.S, w.oversample, w.beta)
    plan = gb.Plan(w.G, w.S, w.oversample, 1, B=2)
    uv = torch.from_numpy(w.uv).cuda()
    wt = torch.from_numpy(w.weights).cuda()

    def loss_of_grid(g):  # FP64 loss from the FP32 grid: sum |FFT(grid) - target|^2
        img = torch.fft.fftshift(torch.fft.ifft2(torch.fft.ifftshift(g.to(torch.complex128)[0]), norm="forward"))
        return torch.sum(torch.abs(img - target) ** 2)

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
        for part, dv in (("re", 1.0 + 0j), ("im", 1j)):
            one.fill_(dv)
            gk.zero_()
            gb.grid(plan, uv[k:k + 1].contiguous(), one, wt[k:k + 1].contiguous(), table, gk)
            lp = float(loss_of_grid(g0 + h * gk))
            lm = float(loss_of_grid(g0 - h * gk))
            fd = (lp - lm) / (2 * h)
            an = grad[k].real if part == "re" else grad[k].imag
            # PyTorch's complex gradient is dL/dRe + i dL/dIm
            err = abs(fd - an) / max(abs(an), 1e-30)
            worst = max(worst, err)
            assert err <= 1e-3, (k, part, fd, an)
    assert worst <= 1e-3
