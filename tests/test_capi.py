"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/gridder.h declares, and rejects bad arguments with
GRID_ERR_INVALID before touching the device."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1605_07023_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("library not built and nvcc unavailable")
        build.build()
    return _lib.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gridder.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ("grid_plan_create", "grid", "degrid", "grid_make_kernel_table", "grid_compute_indices", "grid_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1605_07023_gb300 import _lib
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTS)


def test_invalid_plans_are_rejected_on_the_host(lib):
    from paper_1605_07023_gb300 import _lib
    h = ctypes.c_void_p()
    bad = [(0, 7, 8, 1, 1), (255, 7, 8, 1, 1), (256, 0, 8, 1, 1), (256, 7, 6, 1, 1), (256, 7, 8, 3, 1),
           (256, 7, 8, 1, 0), (256, 7, 8, 1, 9), (8, 9, 8, 1, 1), (65536, 7, 8, 1, 1), (256, 65, 8, 1, 1),
           (256, 7, 512, 1, 1)]
    for args in bad:
        rc = lib.grid_plan_create(ctypes.byref(h), *args)
        assert rc == _lib.GRID_ERR_INVALID, (args, rc)
        assert lib.grid_last_error().decode()
        assert not h.value


def test_null_arguments(lib):
    from paper_1605_07023_gb300 import _lib
    assert lib.grid_plan_create(None, 256, 7, 8, 1, 1) == _lib.GRID_ERR_INVALID
    assert lib.grid(None, 10, None, None, None, None, None, None) == _lib.GRID_ERR_INVALID
    assert lib.degrid(None, 10, None, None, None, None, None) == _lib.GRID_ERR_INVALID
    assert lib.grid_make_kernel_table(0, 8, 16.0, 0, None, None) == _lib.GRID_ERR_INVALID
    assert lib.grid_make_kernel_table(7, 8, 16.0, 0, None, None) == _lib.GRID_ERR_INVALID
    assert lib.grid_make_kernel_table(7, 8, float("nan"), 0, ctypes.c_void_p(16), None) == _lib.GRID_ERR_INVALID
    lib.grid_plan_destroy(None)


def test_desc_init_defaults(lib):
    from paper_1605_07023_gb300 import _lib
    d = _lib.GridPlanDesc()
    lib.grid_plan_desc_init(ctypes.byref(d), 2048, 7, 8, 4, 2)
    assert (d.G, d.S, d.oversample, d.npol, d.Bu, d.Bv) == (2048, 7, 8, 4, 2, 2)
    assert d.precision == 0 and d.schedule == 0 and d.tile_group == 0


def test_newer_entry_points_reject_bad_arguments(lib):
    from paper_1605_07023_gb300 import _lib
    INV = _lib.GRID_ERR_INVALID
    # pipelined host pass, compression and expansion: no plan
    assert lib.grid_degrid_host(None, None, 0, None, None, None, None, None, None, None, None, None, None, None, 0,
                                None) == INV
    assert lib.grid_compress(None, 0, None, None, None, None, None, None, None, None) == INV
    assert lib.degrid_expand(None, 0, None, 0, None, None, None, None) == INV
    # two-shape batches: bad grid side, bad split, and shapes with no kernel
    h = ctypes.c_void_p()
    assert lib.grid_batch_create_ex(ctypes.byref(h), 3, 8, 1, 2, 2, 4, 2, 13, 15, 0, 0, 0) == INV
    assert lib.grid_batch_create_ex(ctypes.byref(h), 1024, 8, 1, 2, 2, 4, 2, 99, 15, 0, 0, 0) == INV
    assert lib.grid_batch_create_ex(ctypes.byref(h), 1024, 8, 1, 2, 2, 8, 8, 13, 15, 0, 0, 0) == _lib.GRID_ERR_UNSUPPORTED
    assert not h.value


def test_schedule_and_tile_threads_checked_on_the_host(lib):
    """Unknown schedules, tile- and lazy-schedule CTA sizes that are not whole warps, and bin widths
    given to a schedule other than the lazy one are rejected before any device call."""
    from paper_1605_07023_gb300 import _lib
    h = ctypes.c_void_p()
    for sched, threads, bins in [(5, 0, 0), (-1, 0, 0), (_lib.SCHED["tile"], 48, 0), (_lib.SCHED["tile"], 100, 0),
                                 (_lib.SCHED["lazy"], 48, 0), (_lib.SCHED["chunked"], 0, 10)]:
        d = _lib.GridPlanDesc()
        lib.grid_plan_desc_init(ctypes.byref(d), 256, 7, 8, 4, 2)
        d.schedule = sched
        d.threads = threads
        d.bin_u = bins
        assert lib.grid_plan_create_ex(ctypes.byref(h), ctypes.byref(d)) == _lib.GRID_ERR_INVALID, (sched, threads, bins)
        assert not h.value
    # tile groups other than 32 and 8, or given to another schedule
    for sched, group in [(_lib.SCHED["tile"], 16), (_lib.SCHED["tile"], -8), (_lib.SCHED["chunked"], 8),
                         (_lib.SCHED["sorted"], 32)]:
        d = _lib.GridPlanDesc()
        lib.grid_plan_desc_init(ctypes.byref(d), 256, 7, 8, 4, 2)
        d.schedule = sched
        d.tile_group = group
        assert lib.grid_plan_create_ex(ctypes.byref(h), ctypes.byref(d)) == _lib.GRID_ERR_INVALID, (sched, group)
        assert not h.value
