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
    cfg = {"all-all": {"cell_scale": 0.5, "dense_min": 0, "split": 1}, "Sc-Sc": {"cell_scale": 0.5, "dense_min": 0, "split": 1}}
    v = bench.stored_traffic("needle2g", cfg)
    # either the stored figure (sources unchanged since the capture) or None; never for another setup
    assert v is None or v > 0
    assert bench.stored_traffic("needle2g", {**cfg, "Sc-Sc": {"cell_scale": 1.0, "dense_min": 0, "split": 0}}) is None
    assert bench.stored_traffic("cylinder200k", cfg) is None


@pytest.mark.parametrize("shares", [1, 3, 7])
def test_small_sample_shares_sum_exactly(orc, shares):
    """The all-core oracle baseline on a small cloud: the centrals of a z-slab sample split in
    shares (one host thread each, every share sees all the slab's neighbours) add up to the
    oracle over the whole sample, histogram for histogram."""
    rng = np.random.default_rng(11)
    n = 6000
    xyz = (rng.random((n, 3)) * np.array([6.0, 6.0, 14.0])).astype(np.float32)
    t = rng.integers(0, 3, n).astype(np.uint8)
    d = (rng.random(n) * 2.0).astype(np.float32)
    wl = dict(bins=(0.0, 0.05, 20), combos=[("x", "all", [0, 2])], ks=[1, 3], dsrf_min=0.5)
    whole = bench.small_sample(wl, (xyz, t, d), 0.6, 1)[0][0]
    ref = orc.spatstat(*whole, "all", [0, 2], 0.5, 0.0, 0.05, 20, [1, 3])
    parts = bench.small_sample(wl, (xyz, t, d), 0.6, shares)[0]
    got = [orc.spatstat(*p, "all", [0, 2], 0.5, 0.0, 0.05, 20, [1, 3]) for p in parts]
    assert ref["n_central"] > 0
    assert sum(g["n_central"] for g in got) == ref["n_central"]
    np.testing.assert_array_equal(sum(g["rdf"] for g in got), ref["rdf"])
    np.testing.assert_array_equal(sum(g["knn"] for g in got), ref["knn"])
    # and the sample's centrals are exactly those of the whole cloud inside the slab
    z = xyz[:, 2]
    z0 = z.min() + 0.5 * (z.max() - z.min()) * 0.4
    z1 = z0 + 0.6 * (z.max() - z.min())
    assert ref["n_central"] == int(((z >= z0) & (z < z1) & (d >= 0.5)).sum())


def test_needle_sample_is_the_middle_of_the_needle(orc, spec, monkeypatch):
    """The large-needle sample generates only lattice layers about mid-height; its ions are the
    full cloud's ions of those layers (same generator), its halo ions are never central."""
    p = spec.needle_params(5.0, 10.0, 16.0, seed=9)
    monkeypatch.setattr(bench, "needle_params", lambda name: p)
    wl = dict(bins=(0.0, 0.01, 100), combos=[("all-all", "all", "all")], ks=[1], dsrf_min=0.5)
    parts, desc = bench.needle_sample("x", wl, 4, 3)
    counts = spec.needle_plan(p)
    off = np.concatenate([[0], np.cumsum(counts)])
    xyz, t, d = spec.needle(p)
    mid = len(counts) // 2
    lo, hi = mid - 2, mid + 2
    core = set(range(off[lo], off[hi]))
    n_core = sum(int(np.count_nonzero(~np.isnan(pd))) for _, _, pd in parts)
    assert n_core == off[hi] - off[lo] == len(core)
    got = sum(orc.spatstat(*pt, "all", "all", 0.5, 0.0, 0.01, 100, [1])["n_central"] for pt in parts)
    assert got == int((d[off[lo]:off[hi]] >= 0.5).sum())


def test_symmetric_pass_test_count_brute_force():
    """The symmetric RDF pass tests every unordered pair of records whose cells are within the
    stencil once: (sum over records of their stencil population - n) / 2, by brute force."""
    rng = np.random.default_rng(8)
    n = 2500
    xyz = (rng.random((n, 3)) * np.array([6.0, 5.0, 7.0])).astype(np.float32)
    t = rng.integers(0, 2, n).astype(np.uint8)
    d = np.full(n, np.nan, np.float32)  # no d_srf filter applies to the record count
    h, stencil = 1.0, 2
    org = xyz.min(axis=0)
    dims = tuple(int(np.floor((xyz[:, a].max() - org[a]) / h)) + 1 for a in range(3))
    info = dict(dims=dims, origin=tuple(float(v) for v in org), cell=h, n_cells=dims[0] * dims[1] * dims[2])
    full = bench.candidate_tests(torch.from_numpy(xyz), torch.from_numpy(t), torch.from_numpy(d), "all", "all", 0.0,
                                 info, stencil, all_records=True)
    c = _cells_np(xyz, org, np.float32(1.0 / h), dims)
    cheb = np.abs(c[:, None, :] - c[None, :, :]).max(axis=2)
    pairs = int(np.triu(cheb <= stencil, k=1).sum())
    assert (full - n) // 2 == pairs and (full - n) % 2 == 0
