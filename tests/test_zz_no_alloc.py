"""grid_patch_static(): gridding for callers that cannot allocate device memory.

Such callers (a real-time pipeline that reserves all of its device memory at
start-up and may not allocate while observing, or a host framework that owns
the device heap through its own allocator) cannot create a plan, because plan
creation and the patch schedule allocate scratch. grid_patch_static() keeps
that scratch in a file-scope device array instead.

The test calls it through the C ABI twice in a row, on two different problems,
so anything stale left in the shared scratch by the first call would show in
the second. Each result is compared, per polarization plane, with the FP64
oracle and with grid() (the plan-based entry point) on the same inputs, within
the tolerance of the other parity tests. A 16-bit case compares it with grid()
and with the oracle fed the same rounded inputs.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _lib():
    from paper_1605_07023_gb300 import _lib as L
    lib = L.load()
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    lib.grid_patch_static.argtypes = [i32, i32, i32, i32, i32, i32, i32, i64, vp, vp, vp, vp, vp, vp]
    lib.grid_patch_static.restype = i32
    lib.grid_patch_static_last_error.argtypes = []
    lib.grid_patch_static_last_error.restype = ctypes.c_char_p
    return lib


PREC = {"f32": 0, "bf16": 1, "f16": 2}


def _inputs(w, precision):
    """Device inputs in the storage format, and the same values upcast exactly for the oracle."""
    t32 = oracle.kb_table(w.S, w.oversample, w.beta).astype(np.float32)
    if precision == "f32":
        vis_d = torch.from_numpy(np.ascontiguousarray(w.vis)).cuda()
        tab_d = torch.from_numpy(t32).cuda()
        vis64, tab64 = w.vis.astype(np.complex128), t32.astype(np.float64)
    else:
        dt = torch.bfloat16 if precision == "bf16" else torch.float16
        v16 = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(w.vis))).to(dt).contiguous()
        t16 = torch.from_numpy(t32).to(dt)
        vis_d, tab_d = v16.cuda(), t16.cuda()
        vis64 = torch.view_as_complex(v16.float().contiguous()).numpy().astype(np.complex128)
        tab64 = t16.float().numpy().astype(np.float64)
    dev = dict(uv=torch.from_numpy(np.ascontiguousarray(w.uv)).cuda(), vis=vis_d,
               wt=torch.from_numpy(np.ascontiguousarray(w.weights)).cuda(), tab=tab_d)
    return dev, vis64, tab64


def _grid_plan(w, B, dev, precision):
    import paper_1605_07023_gb300 as gb
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, Bu=B[0], Bv=B[1], schedule="patch", vis_per_chunk=64,
                   precision=precision)
    ref = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, dev["uv"], dev["vis"], dev["wt"], dev["tab"], ref)
    return ref


def _call_static(lib, w, B, dev, out, precision):
    rc = lib.grid_patch_static(w.G, w.S, w.oversample, w.npol, B[0], B[1], PREC[precision], w.n_vis,
                               dev["uv"].data_ptr(), dev["vis"].data_ptr(), dev["wt"].data_ptr(), dev["tab"].data_ptr(),
                               out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, lib.grid_patch_static_last_error().decode()


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _check(lib, w, B, precision):
    dev, vis64, tab64 = _inputs(w, precision)
    out = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device="cuda")
    _call_static(lib, w, B, dev, out, precision)
    ref = _grid_plan(w, B, dev, precision)
    torch.cuda.synchronize()
    got, via_plan = out.cpu().numpy(), ref.cpu().numpy()
    want, _ = oracle.grid(w.G, w.S, w.oversample, w.uv, vis64, w.weights, tab64)
    for p in range(w.npol):
        assert rel_l2(got[p], want[p]) <= TOL, (w.name, precision, p, "oracle")
        assert rel_l2(got[p], via_plan[p]) <= TOL, (w.name, precision, p, "grid()")


def test_static_scratch_entry_point_matches_oracle_and_grid_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_07023_gb300 import synth
    lib = _lib()
    # two calls in a row on different problems: G=2048 P=4 (4096 patches), then G=256 P=1
    _check(lib, synth.scaled_down(synth.quad_pol(), 300_007), (2, 2), "f32")
    _check(lib, synth.plain_single_pol(), (1, 1), "f32")


def test_static_scratch_entry_point_16bit_storage():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_07023_gb300 import synth
    lib = _lib()
    _check(lib, synth.scaled_down(synth.quad_pol(), 100_003), (2, 2), "bf16")
    _check(lib, synth.scaled_down(synth.quad_pol(), 50_001), (1, 1), "f16")


def test_static_scratch_limit_and_arguments_are_enforced():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib()
    uv = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    vis = torch.zeros((4, 1), dtype=torch.complex64, device="cuda")
    tab = torch.ones((8, 7), dtype=torch.float32, device="cuda")
    g = torch.zeros((1, 256, 256), dtype=torch.complex64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.grid_patch_static(256, 7, 8, 1, 2, 2, 0, 1 << 30, uv.data_ptr(), vis.data_ptr(), None, tab.data_ptr(),
                               g.data_ptr(), st)
    assert rc == -1
    assert b"limit" in lib.grid_patch_static_last_error()
    # an unsupported polarization count is reported as such, before any alignment check
    rc = lib.grid_patch_static(256, 7, 8, 3, 2, 2, 0, 4, uv.data_ptr() + 8, vis.data_ptr(), None, tab.data_ptr(),
                               g.data_ptr(), st)
    assert rc == -2 and b"npol" in lib.grid_patch_static_last_error()
    # weights must be 4-byte aligned, as for grid()
    wt = torch.ones(8, dtype=torch.float32, device="cuda")
    rc = lib.grid_patch_static(256, 7, 8, 1, 2, 2, 0, 4, uv.data_ptr(), vis.data_ptr(), wt.data_ptr() + 2,
                               tab.data_ptr(), g.data_ptr(), st)
    assert rc == -1 and b"weights" in lib.grid_patch_static_last_error()
    torch.cuda.synchronize()
    assert torch.count_nonzero(g).item() == 0
