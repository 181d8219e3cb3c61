"""Host-side counting in bench.py (no GPU): the candidate-test count behind the ALU roofline and
the guard on the stored ncu traffic figure."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402


def _cells_np(P, org, inv_h, dims):
    u = np.floor((P - org).astype(np.float32) * np.float32(inv_h)).astype(np.int64)
    return np.clip(u, 0, np.array(dims) - 1)


@pytest.mark.parametrize("stencil,h", [(1, 2.0), (2, 1.0)])
def test_candidate_tests_brute_force(stencil, h):
    rng = np.random.default_rng(7)
    n = 3000
    xyz = (rng.random((n, 3)) * np.array([9.0, 7.0, 11.0])).astype(np.float32)
    t = rng.integers(0, 3, n).astype(np.uint8)
    d = (rng.random(n) * 3.0).astype(np.float32)
    org = xyz.min(axis=0)
    dims = tuple(int(np.floor((xyz[:, a].max() - org[a]) / h)) + 1 for a in range(3))
    info = dict(dims=dims, origin=tuple(float(v) for v in org), cell=h, n_cells=dims[0] * dims[1] * dims[2])
    got = bench.candidate_tests(torch.from_numpy(xyz), torch.from_numpy(t), torch.from_numpy(d), [1], [1, 2], 1.0,
                                info, stencil)
    inv_h = np.float32(1.0 / h)
    cn = _cells_np(xyz[np.isin(t, [1, 2])], org, inv_h, dims)
    cc = _cells_np(xyz[(t == 1) & (d >= 1.0)], org, inv_h, dims)
    want = sum(int((np.abs(cn - c).max(axis=1) <= stencil).sum()) for c in cc)
    assert got == want > 0


def test_stored_traffic_guard():
    cfg = {"Sc-Sc": {"cell_scale": 1.0, "dense_min": 0}, "Si-Si": {"cell_scale": 1.0, "dense_min": 0}}
    v = bench.stored_traffic("needle8m", cfg)
    # either the stored figure (sources unchanged since the capture) or None; never for another setup
    assert v is None or v > 0
    assert bench.stored_traffic("needle8m", {**cfg, "Sc-Sc": {"cell_scale": 0.5, "dense_min": 0}}) is None
    assert bench.stored_traffic("cylinder200k", cfg) is None


def test_alu_peak():
    peak, mhz = bench.alu_peak_tflops()
    assert peak == pytest.approx(152 * 128 * mhz * 1e6 / 1e12)


@pytest.mark.parametrize("parts", [1, 3, 7])
def test_slab_parts_sum_exactly(orc, parts):
    """The all-core oracle baseline: independent oracle runs over consecutive z-slabs of centrals
    (each with an r_cut halo of neighbours) add up to the oracle over the whole slab, histogram for
    histogram (the halo holds every neighbour within r_cut of a slab's centrals)."""
    rng = np.random.default_rng(11)
    n = 6000
    xyz = (rng.random((n, 3)) * np.array([6.0, 6.0, 14.0])).astype(np.float32)
    t = rng.integers(0, 3, n).astype(np.uint8)
    d = (rng.random(n) * 2.0).astype(np.float32)
    r0, dr, nb = 0.0, 0.05, 20  # stop = 1.0 = the halo
    ks = [1, 3]
    whole = bench.slab_parts(xyz, t, d, 0.6, dr * nb, 1)[0]
    ref = orc.spatstat(*whole, "all", [0, 2], 0.5, r0, dr, nb, ks)
    got = [orc.spatstat(*p, "all", [0, 2], 0.5, r0, dr, nb, ks) for p in bench.slab_parts(xyz, t, d, 0.6, dr * nb, parts)]
    assert ref["n_central"] > 0
    assert sum(g["n_central"] for g in got) == ref["n_central"]
    np.testing.assert_array_equal(sum(g["rdf"] for g in got), ref["rdf"])
    np.testing.assert_array_equal(sum(g["knn"] for g in got), ref["knn"])
    np.testing.assert_array_equal(sum(np.asarray(g["not_found"]) for g in got), np.asarray(ref["not_found"]))
