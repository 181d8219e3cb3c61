"""Failure detection on the host (no GPU): an injected device-allocation failure makes the
allocating entry points return PS_ERR_OOM with nothing left allocated, before any other CUDA
call; the debug hooks refuse bad arguments."""
import ctypes

import pytest

import paper_2004_05188_gb300 as ps

OK, INVALID_ARG, OOM = 0, 1, 3


@pytest.fixture(scope="module")
def L():
    from paper_2004_05188_gb300 import _build

    _build.build()
    return ps.lib()


def test_injected_grid_allocation_failure(L):
    live = L.ps_debug_live_allocs()
    assert L.ps_debug_fail_alloc(1) == OK
    h = ctypes.c_void_p(1234)
    opts = ps.GridOpts(ctypes.sizeof(ps.GridOpts), 1.0, 0, 0)
    assert L.ps_grid_create(1000, ctypes.byref(opts), ctypes.byref(h)) == OOM
    assert not h.value  # no handle escapes
    assert "out of memory" in L.ps_last_error().decode()
    assert L.ps_debug_live_allocs() == live
    assert L.ps_debug_fail_alloc(0) == OK


def test_injected_failure_inside_batch_create(L):
    """The batch allocates one grid per ROI first: the first allocation fails, the batch
    cleans up and returns PS_ERR_OOM."""
    live = L.ps_debug_live_allocs()
    ds = (ps.Dataset * 2)(ps.Dataset(None, None, None, 0), ps.Dataset(None, None, None, 0))
    sw = ps.Sweep()
    sw.struct_size = ctypes.sizeof(ps.Sweep)
    sw.bins = ps.Bins(0.0, 0.01, 100)
    sw.n_rmax, sw.rmax_bins[0] = 1, 100
    sw.n_dsrf, sw.dsrf_min[0] = 1, 0.0
    sw.n_pairs = 1
    for w in range(4):
        sw.ctr_mask[0][w] = sw.nbr_mask[0][w] = 0xFFFFFFFFFFFFFFFF
    sw.k_max, sw.cell_scale = 4, 1.0
    h = ctypes.c_void_p()
    assert L.ps_debug_fail_alloc(1) == OK
    assert L.ps_batch_create(ds, 2, ctypes.byref(sw), ctypes.byref(h)) == OOM
    assert not h.value
    assert L.ps_debug_live_allocs() == live
    L.ps_debug_fail_alloc(0)


def test_debug_hook_arguments(L):
    assert L.ps_debug_fail_alloc(-1) == INVALID_ARG
    assert L.ps_debug_wait_selftest(1000, None, None) == INVALID_ARG
    work = ctypes.c_void_p(16)  # never dereferenced: the limit is refused first
    assert L.ps_debug_wait_selftest(3_000_000_000, work, None) == INVALID_ARG
    assert "2 s" in L.ps_last_error().decode()
