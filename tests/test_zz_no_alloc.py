"""grid_patch_static(): gridding for callers that cannot allocate device memory.

Such callers (a real-time pipeline that reserves all device memory at
start-up, code running inside a CUDA-graph stream capture, a host framework
that owns the device heap) cannot create a plan, because plan creation and
the patch schedule allocate scratch. grid_patch_static() keeps that scratch in
a file-scope device array instead. This test calls it through the C ABI twice
in a row, on two different problems, so anything stale left in the shared
scratch by the first call would show in the second. Each time it compares the
result with grid() (the plan-based entry point, patch schedule) on the same
inputs, within the same tolerance as the other parity tests.

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


def _problem(w, B):
    import paper_1605_07023_gb300 as gb
    t32 = oracle.kb_table(w.S, w.oversample, w.beta).astype(np.float32)
    dev = dict(uv=torch.from_numpy(np.ascontiguousarray(w.uv)).cuda(),
               vis=torch.from_numpy(np.ascontiguousarray(w.vis)).cuda(),
               wt=torch.from_numpy(np.ascontiguousarray(w.weights)).cuda(),
               tab=torch.from_numpy(t32).cuda())
    plan = gb.Plan(w.G, w.S, w.oversample, w.npol, Bu=B[0], Bv=B[1], schedule="patch", vis_per_chunk=64)
    ref = torch.zeros((w.npol, w.G, w.G), dtype=torch.complex64, device="cuda")
    gb.grid(plan, dev["uv"], dev["vis"], dev["wt"], dev["tab"], ref)
    return dev, ref


def _call_static(lib, w, B, dev, out):
    rc = lib.grid_patch_static(w.G, w.S, w.oversample, w.npol, B[0], B[1], 0, w.n_vis, dev["uv"].data_ptr(),
                               dev["vis"].data_ptr(), dev["wt"].data_ptr(), dev["tab"].data_ptr(), out.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert rc == 0, lib.grid_patch_static_last_error().decode()


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_static_scratch_entry_point_matches_grid_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_07023_gb300 import synth
    lib = _lib()
    cases = [(synth.scaled_down(synth.quad_pol(), 300_007), (2, 2)),        # G=2048, P=4, 4096 patches
             (synth.plain_single_pol(), (1, 1))]                           # G=256, P=1, fewer chunks and patches
    for w, B in cases:
        dev, ref = _problem(w, B)
        out = torch.zeros_like(ref)
        _call_static(lib, w, B, dev, out)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        for p in range(w.npol):
            assert rel_l2(got[p], want[p]) <= TOL, (w.name, p)


def test_static_scratch_limit_is_enforced():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = _lib()
    uv = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    vis = torch.zeros((4, 1), dtype=torch.complex64, device="cuda")
    tab = torch.ones((8, 7), dtype=torch.float32, device="cuda")
    g = torch.zeros((1, 256, 256), dtype=torch.complex64, device="cuda")
    rc = lib.grid_patch_static(256, 7, 8, 1, 2, 2, 0, 1 << 30, uv.data_ptr(), vis.data_ptr(), None, tab.data_ptr(),
                               g.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == -1
    assert b"limit" in lib.grid_patch_static_last_error()
    assert torch.count_nonzero(g).item() == 0
