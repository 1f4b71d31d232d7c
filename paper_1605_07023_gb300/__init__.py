"""GB300-native convolutional gridding with Romein's sliding window and thread coarsening.

A thin binding over the C ABI in ``include/gridder.h``. The functions keep the
ABI's names and only marshal arguments: tensors must already live on the CUDA
device, and all the work runs in the library's CUDA kernels on the caller's
current stream. There is no CPU path; if the library is not built, every call
raises RuntimeError.

Layouts (see the header for the full contract):
  - uv: [n, 2] float64, in grid pixels relative to the centre.
  - vis: [n, P] complex64. For 16-bit storage, [n, P, 2] bfloat16 / float16.
  - weights: [n] float32 or None.
  - kernel_table: [O, S] float32 / bfloat16 / float16.
  - grid: [P, G, G] complex64.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import GridderError, PREC, SCHED

__all__ = ["Plan", "BatchPlan", "grid_plan_create", "grid_plan_create_ex", "grid", "degrid", "degrid_weighted", "grid_make_kernel_table",
           "grid_compute_indices", "device_info", "tap_form", "measure_fma_peak", "GridderError"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dptr(t, name: str, dtype=None, ndim=None) -> int:
    torch = _torch()
    if t is None:
        return 0
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimensions, has {t.dim()}")
    return t.data_ptr()


class Plan:
    """Owns one grid_plan_t (destroyed on close() or garbage collection).

    schedule: "chunked" (fixed visibilities per team, global flushes), "patch" (chunks binned by
    grid patch, flushes into a shared-memory window), "tile" (grids as "chunked"; degrids by
    tile gather, one warp per tile_group = 32 or 8 visibilities, threads a multiple of 32), or "lazy" (grids with a
    bin of bin_u x bin_v cells, wider than the paper's, whose box moves only when the footprint
    leaves it; degrids as "chunked").
    """

    def __init__(self, G: int, S: int, oversample: int, npol: int, B: int = 1, Bu: int | None = None,
                 Bv: int | None = None, vis_per_chunk: int = 0, threads: int = 0, precision: str = "f32",
                 schedule: str = "chunked", patch: int = 0, bin_u: int = 0, bin_v: int = 0, tile_group: int = 0):
        lib = _lib.load()
        d = _lib.GridPlanDesc()
        lib.grid_plan_desc_init(ctypes.byref(d), G, S, oversample, npol, B)
        d.Bu = B if Bu is None else Bu
        d.Bv = B if Bv is None else Bv
        d.vis_per_chunk = vis_per_chunk
        d.threads = threads
        d.precision = PREC[precision]
        d.schedule = SCHED[schedule]
        d.patch = patch
        d.bin_u = bin_u
        d.bin_v = bin_v
        d.tile_group = tile_group
        h = ctypes.c_void_p()
        _lib.check(lib.grid_plan_create_ex(ctypes.byref(h), ctypes.byref(d)))
        self._h = h
        self.G, self.S, self.oversample, self.npol = G, S, oversample, npol
        self.precision = precision
        self.schedule = schedule

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("plan is closed")
        return self._h

    def describe(self) -> dict:
        d = _lib.GridPlanDesc()
        bu, bv, ts = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(_lib.load().grid_plan_describe(self.handle, ctypes.byref(d), ctypes.byref(bu), ctypes.byref(bv),
                                                  ctypes.byref(ts)))
        out = {n: getattr(d, n) for n, _ in _lib.GridPlanDesc._fields_}
        out.update(bin_u=bu.value, bin_v=bv.value, team_size=ts.value, gridder=self.gridder())
        return out

    def gridder(self) -> str:
        """Name of the kernel grid() launches: chunked, patch, lazy, sorted or sorted-wide."""
        return _lib.load().grid_plan_gridder(self.handle).decode()

    def skipped(self, reset: bool = False) -> int:
        v = ctypes.c_int64()
        _lib.check(_lib.load().grid_plan_skipped(self.handle, ctypes.byref(v), int(reset)))
        return v.value

    def status(self, reset: bool = False) -> int:
        """Status flags of the plan's gridding calls (bit 0: a bulk copy of records timed out)."""
        v = ctypes.c_uint()
        _lib.check(_lib.load().grid_plan_status(self.handle, ctypes.byref(v), int(reset)))
        return v.value

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _lib.load().grid_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # convenience wrappers
    def grid(self, uv, vis, weights, kernel_table, grid_out, stream=None):
        return grid(self, uv, vis, weights, kernel_table, grid_out, stream)

    def degrid(self, uv, grid_in, kernel_table, vis_out=None, stream=None):
        return degrid(self, uv, grid_in, kernel_table, vis_out, stream)


def grid_plan_create(G: int, S: int, oversample: int, npol: int, B: int = 1) -> Plan:
    return Plan(G, S, oversample, npol, B)


def grid_plan_create_ex(**kw) -> Plan:
    return Plan(**kw)


def _vis_dtype(plan: Plan):
    torch = _torch()
    return {"f32": torch.complex64, "bf16": torch.bfloat16, "f16": torch.float16}[plan.precision]


def grid(plan: Plan, uv, vis, weights, kernel_table, grid_out, stream=None):
    """grid(): accumulate the visibilities into grid_out ([P, G, G] complex64). Returns grid_out."""
    torch = _torch()
    n = uv.shape[0]
    pu = _dptr(uv, "uv", torch.float64, 2)
    pv = _dptr(vis, "vis", _vis_dtype(plan))
    pw = _dptr(weights, "weights", torch.float32, 1)
    pt = _dptr(kernel_table, "kernel_table", (torch.float32, torch.bfloat16, torch.float16), 2)
    pg = _dptr(grid_out, "grid", torch.complex64, 3)
    if vis.shape[0] != n or (weights is not None and weights.shape[0] != n):
        raise ValueError("uv, vis and weights must have the same length")
    if tuple(grid_out.shape) != (plan.npol, plan.G, plan.G):
        raise ValueError(f"grid must be [{plan.npol}, {plan.G}, {plan.G}]")
    _lib.check(_lib.load().grid(plan.handle, n, pu, pv, pw or None, pt, pg, _stream_ptr(stream)))
    return grid_out


def degrid(plan: Plan, uv, grid_in, kernel_table, vis_out=None, stream=None):
    """degrid(): visibilities [n, P] complex64 from grid_in (overwrites vis_out). Returns vis_out."""
    return degrid_weighted(plan, uv, grid_in, kernel_table, None, vis_out, stream)


def degrid_weighted(plan: Plan, uv, grid_in, kernel_table, weights, vis_out=None, stream=None):
    """degrid_weighted(): w_n * degrid(grid_in)[n], the adjoint of weighted grid(). weights None = degrid()."""
    torch = _torch()
    n = uv.shape[0]
    if vis_out is None:
        vis_out = torch.empty((n, plan.npol), dtype=torch.complex64, device=uv.device)
    pu = _dptr(uv, "uv", torch.float64, 2)
    pg = _dptr(grid_in, "grid", torch.complex64, 3)
    pt = _dptr(kernel_table, "kernel_table", (torch.float32, torch.bfloat16, torch.float16), 2)
    po = _dptr(vis_out, "vis", torch.complex64, 2)
    pw = _dptr(weights, "weights", torch.float32, 1)
    if tuple(grid_in.shape) != (plan.npol, plan.G, plan.G):
        raise ValueError(f"grid must be [{plan.npol}, {plan.G}, {plan.G}]")
    if weights is not None and weights.shape[0] != n:
        raise ValueError("weights must have one entry per visibility")
    _lib.check(_lib.load().degrid_weighted(plan.handle, n, pu, pg, pt, pw or None, po, _stream_ptr(stream)))
    return vis_out


def grid_compress(plan: Plan, uv, vis, weights=None, stream=None, out=None, sync: bool = True):
    """grid_compress(): merge runs of adjacent visibilities on one oversampled-grid point.

    Returns ``(uv_c [m, 2] float64, vis_c [m, P] complex64, run_of [n] int64)``. ``vis_c`` holds the
    weighted sums (grid it with weights=None and an FP32 plan); ``run_of[k]`` is the run of visibility k.
    Reading the run count m back synchronises with the stream. ``out`` = (uv_c, vis_c, run_of, n_out)
    supplies the full-size output buffers. With ``sync=False`` nothing is read back: the call returns
    the untrimmed buffers and the device tensor n_out holding m.
    """
    torch = _torch()
    n = uv.shape[0]
    pu = _dptr(uv, "uv", torch.float64, 2)
    pv = _dptr(vis, "vis", _vis_dtype(plan))
    pw = _dptr(weights, "weights", torch.float32, 1)
    if vis.shape[0] != n or (weights is not None and weights.shape[0] != n):
        raise ValueError("uv, vis and weights must have the same length")
    if out is None:
        out = (torch.empty((n, 2), dtype=torch.float64, device=uv.device),
               torch.empty((n, plan.npol), dtype=torch.complex64, device=uv.device),
               torch.empty(n, dtype=torch.int64, device=uv.device),
               torch.zeros(1, dtype=torch.int64, device=uv.device))
    uv_c, vis_c, run_of, n_out = out
    if uv_c.shape[0] < n or vis_c.shape[0] < n or run_of.shape[0] < n:
        raise ValueError("output buffers need room for n records")
    _lib.check(_lib.load().grid_compress(plan.handle, n, pu, pv, pw or None, _dptr(uv_c, "uv_c", torch.float64, 2),
                                         _dptr(vis_c, "vis_c", torch.complex64, 2), _dptr(run_of, "run_of", torch.int64, 1),
                                         _dptr(n_out, "n_out", torch.int64, 1), _stream_ptr(stream)))
    if not sync:
        return uv_c, vis_c, run_of, n_out
    m = int(n_out.item())
    return uv_c[:m], vis_c[:m], run_of[:n]


def degrid_expand(plan: Plan, run_of, vis_c, weights=None, vis_out=None, stream=None):
    """degrid_expand(): vis_out[k] = w_k * vis_c[run_of[k]] (the degridded value of each merged record's members)."""
    torch = _torch()
    n = run_of.shape[0]
    if vis_out is None:
        vis_out = torch.empty((n, plan.npol), dtype=torch.complex64, device=run_of.device)
    pr = _dptr(run_of, "run_of", torch.int64, 1)
    pc = _dptr(vis_c, "vis_c", torch.complex64, 2) if vis_c.shape[0] > 0 else 0
    pw = _dptr(weights, "weights", torch.float32, 1)
    po = _dptr(vis_out, "vis_out", torch.complex64, 2)
    if weights is not None and weights.shape[0] != n:
        raise ValueError("weights must have one entry per visibility")
    _lib.check(_lib.load().degrid_expand(plan.handle, n, pr, int(vis_c.shape[0]), pc or None, pw or None, po,
                                         _stream_ptr(stream)))
    return vis_out


def _hptr(t, name: str, dtype=None) -> int:
    torch = _torch()
    if t is None:
        return 0
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} has dtype {t.dtype}, expected {dtype}")
    return t.data_ptr()


def grid_degrid_host(gplan: Plan, dplan: Plan, uv_host, vis_host, weights_host, kernel_table, grid, vis_out_host,
                     grid_host=None, work=None, chunk: int = 0, stream=None):
    """grid_degrid_host(): zero the grid, grid and degrid from HOST (pinned) buffers with the copies overlapped.

    ``work`` = (uv_dev, vis_dev, weights_dev, vis_out_dev) device buffers with room for n visibilities
    (allocated here if None). Fills vis_out_host (and grid_host if given) once the stream reaches the end
    of the call. Returns vis_out_host.
    """
    torch = _torch()
    n = uv_host.shape[0]
    dev = grid.device
    if work is None:
        work = (torch.empty((n, 2), dtype=torch.float64, device=dev), torch.empty_like(vis_host, device=dev),
                None if weights_host is None else torch.empty_like(weights_host, device=dev),
                torch.empty((n, gplan.npol), dtype=torch.complex64, device=dev))
    uv_d, vis_d, wt_d, out_d = work
    if vis_host.shape[0] != n or (weights_host is not None and weights_host.shape[0] != n) or vis_out_host.shape[0] != n:
        raise ValueError("host buffers must have one row per visibility")
    if tuple(grid.shape) != (gplan.npol, gplan.G, gplan.G):
        raise ValueError(f"grid must be [{gplan.npol}, {gplan.G}, {gplan.G}]")
    args = (gplan.handle, dplan.handle, n, _hptr(uv_host, "uv_host", torch.float64),
            _hptr(vis_host, "vis_host", _vis_dtype(gplan)), _hptr(weights_host, "weights_host", torch.float32) or None,
            _dptr(uv_d, "uv_dev", torch.float64, 2), _dptr(vis_d, "vis_dev", _vis_dtype(gplan)),
            _dptr(wt_d, "weights_dev", torch.float32, 1) or None, _dptr(out_d, "vis_out_dev", torch.complex64, 2),
            _dptr(kernel_table, "kernel_table", (torch.float32, torch.bfloat16, torch.float16), 2),
            _dptr(grid, "grid", torch.complex64, 3), _hptr(vis_out_host, "vis_out_host", torch.complex64),
            _hptr(grid_host, "grid_host", torch.complex64) or None, int(chunk), _stream_ptr(stream))
    _lib.check(_lib.load().grid_degrid_host(*args))
    return vis_out_host


def grid_degrid_host_steps(gplan: Plan, dplan: Plan, steps, kernel_table, grid, work=None, chunk: int = 0, stream=None):
    """grid_degrid_host_steps(): several grid + degrid passes from pinned host buffers, pipelined across steps.

    steps: list of dicts with host tensors uv, vis, weights (or None), vis_out, grid_out (or None); every step
    has the same visibility count. work: two tuples (uv_dev, vis_dev, weights_dev, vis_out_dev), allocated here
    if None. The host outputs are complete once the stream reaches the end of the call.
    """
    torch = _torch()
    if not steps:
        return
    n = steps[0]["uv"].shape[0]
    dev = grid.device
    if work is None:
        s0 = steps[0]
        work = [(torch.empty((n, 2), dtype=torch.float64, device=dev), torch.empty_like(s0["vis"], device=dev),
                 None if s0["weights"] is None else torch.empty_like(s0["weights"], device=dev),
                 torch.empty((n, gplan.npol), dtype=torch.complex64, device=dev)) for _ in range(2)]
    arr = (_lib.GridHostStep * len(steps))()
    for i, st in enumerate(steps):
        if st["uv"].shape[0] != n or st["vis"].shape[0] != n or st["vis_out"].shape[0] != n:
            raise ValueError("every step must have the same number of visibilities")
        arr[i] = _lib.GridHostStep(_hptr(st["uv"], "uv", torch.float64), _hptr(st["vis"], "vis", _vis_dtype(gplan)),
                                   _hptr(st["weights"], "weights", torch.float32) or None,
                                   _hptr(st["vis_out"], "vis_out", torch.complex64),
                                   _hptr(st.get("grid_out"), "grid_out", torch.complex64) or None)
    P2 = ctypes.c_void_p * 2
    uv_d = P2(*[_dptr(wk[0], "uv_dev", torch.float64, 2) for wk in work])
    vis_d = P2(*[_dptr(wk[1], "vis_dev", _vis_dtype(gplan)) for wk in work])
    wt_d = None if work[0][2] is None else P2(*[_dptr(wk[2], "weights_dev", torch.float32, 1) for wk in work])
    out_d = P2(*[_dptr(wk[3], "vis_out_dev", torch.complex64, 2) for wk in work])
    _lib.check(_lib.load().grid_degrid_host_steps(
        gplan.handle, dplan.handle, len(steps), arr, n, uv_d, vis_d, wt_d, out_d,
        _dptr(kernel_table, "kernel_table", (torch.float32, torch.bfloat16, torch.float16), 2),
        _dptr(grid, "grid", torch.complex64, 3), int(chunk), _stream_ptr(stream)))


def grid_make_kernel_table(S: int, oversample: int, beta: float, precision: str = "f32", device=None, stream=None):
    """Oversampled Kaiser-Bessel table [O, S], computed on the device in FP64 and rounded once."""
    torch = _torch()
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[precision]
    out = torch.empty((oversample, S), dtype=dt, device=device or "cuda")
    _lib.check(_lib.load().grid_make_kernel_table(S, oversample, float(beta), PREC[precision], out.data_ptr(),
                                                  _stream_ptr(stream)))
    return out


def grid_compute_indices(plan: Plan, uv, stream=None):
    """(cell [n, 2] int32, sub [n, 2] int32) as the kernels compute them; -1 marks a skipped visibility."""
    torch = _torch()
    n = uv.shape[0]
    cell = torch.empty((n, 2), dtype=torch.int32, device=uv.device)
    sub = torch.empty((n, 2), dtype=torch.int32, device=uv.device)
    _lib.check(_lib.load().grid_compute_indices(plan.handle, n, _dptr(uv, "uv", torch.float64, 2), cell.data_ptr(),
                                                sub.data_ptr(), _stream_ptr(stream)))
    return cell, sub


def device_info() -> dict:
    sms, lanes, clk = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _lib.check(_lib.load().grid_device_info(ctypes.byref(sms), ctypes.byref(lanes), ctypes.byref(clk)))
    return dict(sm_count=sms.value, fma_lanes_per_sm=lanes.value, max_clock_khz=clk.value)


TAP_FORMS = ("product", "factor_v", "factor_u")


def measure_fma_peak(iters: int = 4096, stream=None) -> float:
    """grid_measure_fma_peak(): the device's measured FP32 FMA rate in TFLOP/s (synchronises)."""
    v = ctypes.c_double()
    _lib.check(_lib.load().grid_measure_fma_peak(int(iters), ctypes.byref(v), _stream_ptr(stream)))
    return v.value


def tap_form(Bu: int, Bv: int, npol: int) -> tuple[str, int]:
    """How the kernels for a Bu x Bv block form the tap products (Sec. 6 remark), and their
    multiplications per visibility per block (grid_tap_form in the C ABI; host only)."""
    form, mults = ctypes.c_int(), ctypes.c_int()
    _lib.check(_lib.load().grid_tap_form(Bu, Bv, npol, ctypes.byref(form), ctypes.byref(mults)))
    return TAP_FORMS[form.value], mults.value


class BatchPlan:
    """Batched gridding of many grids in one persistent launch (grid_batch_* in the C ABI).

    items: list of dicts with keys uv, vis, weights (or None), table, grid, S,
    all CUDA tensors (see grid()). Tensors must stay alive while the batch is
    executed. execute() enqueues one kernel per block shape on the current
    stream and can be captured in a CUDA graph.
    """

    def __init__(self, G: int, oversample: int, npol: int, Bu: int = 2, Bv: int = 2, max_S: int = 15,
                 precision: str = "f32", vis_per_chunk: int = 0, threads: int = 0, Bu2: int | None = None,
                 Bv2: int | None = None, S_split: int = 0):
        """(Bu2, Bv2, S_split): items with S >= S_split use blocks of Bu2 x Bv2 (grid_batch_create_ex)."""
        lib = _lib.load()
        h = ctypes.c_void_p()
        Bu2 = Bu if Bu2 is None else Bu2
        Bv2 = Bv if Bv2 is None else Bv2
        _lib.check(lib.grid_batch_create_ex(ctypes.byref(h), G, oversample, npol, Bu, Bv, Bu2, Bv2, S_split, max_S,
                                            PREC[precision], vis_per_chunk, threads), batch=True)
        self._h = h
        self.G, self.oversample, self.npol, self.precision = G, oversample, npol, precision
        self._keep = []

    def set(self, items) -> None:
        torch = _torch()
        arr = (_lib.GridBatchItem * max(1, len(items)))()
        keep = []
        for k, it in enumerate(items):
            n = it["uv"].shape[0]
            arr[k].n_vis = n
            arr[k].uv = _dptr(it["uv"], "uv", torch.float64, 2) or None
            arr[k].vis = _dptr(it["vis"], "vis", _vis_dtype(self)) or None
            arr[k].weights = _dptr(it.get("weights"), "weights", torch.float32, 1) or None
            arr[k].kernel_table = _dptr(it["table"], "kernel_table", (torch.float32, torch.bfloat16, torch.float16), 2) or None
            g = it["grid"]
            if tuple(g.shape) != (self.npol, self.G, self.G):
                raise ValueError("each grid must be [P, G, G]")
            arr[k].grid = _dptr(g, "grid", torch.complex64, 3) or None
            arr[k].S = int(it["S"])
            keep.append(it)
        _lib.check(_lib.load().grid_batch_set(self.handle, len(items), arr), batch=True)
        self._keep = keep

    def execute(self, stream=None) -> None:
        _lib.check(_lib.load().grid_batch_execute(self.handle, _stream_ptr(stream)), batch=True)

    def describe(self) -> dict:
        t, u, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(_lib.load().grid_batch_describe(self.handle, ctypes.byref(t), ctypes.byref(u), ctypes.byref(c)),
                   batch=True)
        return dict(threads=t.value, units=u.value, ctas=c.value)

    def skipped(self, reset: bool = False) -> int:
        v = ctypes.c_int64()
        _lib.check(_lib.load().grid_batch_skipped(self.handle, ctypes.byref(v), int(reset)), batch=True)
        return v.value

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("batch plan is closed")
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            _lib.load().grid_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
