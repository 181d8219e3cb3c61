"""Failure detection on the GPU, without faulting it.

* The library's bounded device waits (the look-back of the single-pass scans, the mbarrier of
  the bulk copies) run on events that never happen, with a 2 ms limit: both report
  PS_ERR_TIMEOUT, the call returns, and the context stays usable (an exact query afterwards
  still equals the oracle).
* Every device allocation of ps_batch_create is made to fail in turn (host-side injection):
  each time the call returns PS_ERR_OOM and frees everything it had allocated (the library's
  live-allocation count and the device's free memory return to where they were)."""
import ctypes
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2004_05188_gb300 as ps

    return ps


def test_bounded_waits_time_out_and_the_context_survives(ps, orc, spec):
    L = ps.lib()
    work = torch.full((4,), 7, dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    assert L.ps_debug_wait_selftest(2_000_000, ctypes.c_void_p(work.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    w = work.cpu().numpy()
    assert (w[2] & 0xFFFFFFFF) == 5 and w[3] == 5, w  # PS_ERR_TIMEOUT from both waits
    assert dt < 1.0
    # the context is intact: an exact query after the timed-out waits
    xyz, t, d = spec.cylinder(61, 20_000, 5.0, 8.0)
    X, T, D = (torch.from_numpy(a).cuda() for a in (xyz, t, d))
    bins = ps.bins_from_spec(0.0, 0.01, 1.5)
    g = ps.Grid(X.shape[0]).build(X, T, "all", 1.5)
    out = ps.spatstat(g, D, "all", 1.0, bins, [3])
    ref = orc.spatstat(xyz, t, d, "all", "all", 1.0, *bins, [3])
    np.testing.assert_array_equal(out["rdf"].cpu().numpy().astype(np.uint64), ref["rdf"])
    np.testing.assert_array_equal(out["knn"].cpu().numpy().astype(np.uint64), ref["knn"])
    g.close()


def test_every_batch_allocation_failure_is_clean(ps, spec):
    L = ps.lib()
    rois = []
    for i, n in enumerate((3000, 5000, 8000)):
        xyz, t, d = spec.cylinder(70 + i, n, 4.0, 6.0)
        rois.append(tuple(torch.from_numpy(a).cuda() for a in (xyz, t, d)))
    args = ((0.0, 0.01, 100), [50, 100], [0.0, 1.0], [("all", "all"), ([1], [0])], 5)
    torch.cuda.synchronize()
    live0 = L.ps_debug_live_allocs()
    free0 = torch.cuda.mem_get_info()[0]
    n_allocs = len(rois) + 5  # one grid per ROI, then the batch's own arrays
    for nth in range(1, n_allocs + 1):
        assert L.ps_debug_fail_alloc(nth) == 0
        with pytest.raises(ps.PSError) as ei:
            ps.Batch(rois, *args)
        assert ei.value.code == 3, (nth, str(ei.value))
        assert L.ps_debug_live_allocs() == live0, nth
    L.ps_debug_fail_alloc(0)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 64 << 20
    b = ps.Batch(rois, *args)  # and with no injection the same call succeeds
    assert L.ps_debug_live_allocs() == live0 + n_allocs
    out = b.run()
    torch.cuda.synchronize()
    assert int(out[..., -(4 + 2 * 5) + 3].abs().sum().item()) == 0  # no device-side status
    b.close()
    assert L.ps_debug_live_allocs() == live0


def test_injected_grid_failure_through_the_binding(ps):
    L = ps.lib()
    live0 = L.ps_debug_live_allocs()
    L.ps_debug_fail_alloc(1)
    with pytest.raises(ps.PSError) as ei:
        ps.Grid(10_000)
    assert ei.value.code == 3
    L.ps_debug_fail_alloc(0)
    g = ps.Grid(10_000)
    assert L.ps_debug_live_allocs() == live0 + 1
    g.close()
    assert L.ps_debug_live_allocs() == live0
