"""The allocation-free entry point ps_spatstat_static, through the C ABI.

It serves callers that cannot allocate device memory while they run
(applications that give all device memory to their own pool at start-up, loops
that must not block on the device-wide synchronisation of cudaMalloc/cudaFree).
Its output must equal that of the allocating path (ps_build_grid +
ps_spatstat) bit for bit, on consecutive calls that share its static scratch.
This file is collected last so that a failure here leaves every other test run.
"""
import ctypes

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


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _static_call(ps, X, T, D, nbr, r_cut, ctr, dmin, bins, ks):
    L = ps.lib()
    nb, nk, n = bins[2], len(ks), X.shape[0]
    out = dict(rdf=torch.full((nb,), -1, dtype=torch.int64, device="cuda"),
               knn=torch.full((nk, nb), -1, dtype=torch.int64, device="cuda"),
               meta=torch.full((4 + 2 * nk,), -1, dtype=torch.int64, device="cuda"),
               kth=torch.full((nk, n), float("nan"), dtype=torch.float32, device="cuda"),
               nw=torch.full((n,), -1, dtype=torch.int32, device="cuda"))
    ks_a = np.ascontiguousarray(ks, np.uint32)
    mn, mc = ps.type_mask(nbr), ps.type_mask(ctr)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.ps_spatstat_static(_p(X), _p(T), _p(D), n, mn.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(r_cut),
                              mc.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(dmin), ps.Bins(*bins),
                              ks_a.ctypes.data_as(ctypes.c_void_p), nk, _p(out["rdf"]), _p(out["knn"]),
                              _p(out["meta"]), _p(out["kth"]), _p(out["nw"]), stream)
    assert rc == 0, ps.lib().ps_last_error()
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _alloc_call(ps, X, T, D, nbr, r_cut, ctr, dmin, bins, ks):
    g = ps.Grid(X.shape[0]).build(X, T, nbr, r_cut)
    o = ps.spatstat(g, D, ctr, dmin, bins, ks, per_central=True)
    torch.cuda.synchronize()
    res = dict(rdf=o["rdf"].cpu().numpy(), knn=o["knn"].cpu().numpy(), meta=o["meta"].cpu().numpy(),
               kth=o["kth_d2"].cpu().numpy(), nw=o["n_within"].cpu().numpy())
    g.close()
    return res


def test_static_scratch_matches_allocating_path_on_consecutive_calls(ps, spec):
    cases = [
        (spec.cylinder(31, 120_000, 9.0, 12.0), "all", 2.0, "all", 1.0, (0.0, 0.01, 200), [1, 4]),
        (spec.cube(32, 30_000, 10.0, (0.9, 0.1)), [1], 1.5, [1], 0.5, (0.0, 0.02, 75), [2, 7]),
    ]
    for (xyz, t, d), nbr, r_cut, ctr, dmin, bins, ks in cases:
        X, T, D = (torch.from_numpy(a).cuda() for a in (xyz, t, d))
        ref = _alloc_call(ps, X, T, D, nbr, r_cut, ctr, dmin, bins, ks)
        got = _static_call(ps, X, T, D, nbr, r_cut, ctr, dmin, bins, ks)
        assert got["meta"][3] == 0 and got["meta"][0] > 0
        for k in ("rdf", "knn", "meta", "nw"):
            np.testing.assert_array_equal(got[k], ref[k])
        np.testing.assert_array_equal(np.nan_to_num(got["kth"], nan=-1.0), np.nan_to_num(ref["kth"], nan=-1.0))


def test_static_rejects_too_many_ions(ps):
    n = ps.STATIC_MAX_IONS + 1
    X = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    T = torch.zeros(n, dtype=torch.uint8, device="cuda")
    meta = torch.zeros(6, dtype=torch.int64, device="cuda")
    m = ps.type_mask("all")
    ks = np.array([1], np.uint32)
    rc = ps.lib().ps_spatstat_static(_p(X), _p(T), None, n, m.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(1.0),
                                     m.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(0.0), ps.Bins(0.0, 0.1, 10),
                                     ks.ctypes.data_as(ctypes.c_void_p), 1, None, _p(meta), _p(meta), None, None, None)
    assert rc == 7
    assert b"PS_STATIC_MAX_IONS" in ps.lib().ps_last_error()
