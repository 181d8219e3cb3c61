"""Host-side counting in bench.py (no GPU): the candidate-test count behind the ALU roofline and
the guard on the stored ncu traffic figure."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402


def _cells_np(P, org, inv_h, dims):
    u = np.floor((P - org).astype(np.float32) * np.float32(inv_h)).astype(np.int64)
    return np.clip(u, 0, np.array(dims) - 1)


def _kept(dc, cs):
    """Cell offsets the exact query searches: the gap (|d| - 1 cells per axis, on the cell-edge
    bound r_cut cs (1 + 2^-10)) below r_cut (1 + 2^-20); every offset when cs is None."""
    if cs is None:
        return np.ones(dc.shape[:-1], bool)
    m = np.maximum(np.abs(dc) - 1, 0).astype(np.float64)
    f = float(np.float32(cs)) * (1 + 2.0**-10)
    return (m**2).sum(axis=-1) * f * f < (1 + 2.0**-20) ** 2


@pytest.mark.parametrize("stencil,h,cs", [(1, 2.0, None), (2, 1.0, None), (2, 1.0, 0.5), (2, 1.0, 0.75),
                                          (3, 0.7, 1 / 3)])
def test_candidate_tests_brute_force(stencil, h, cs):
    rng = np.random.default_rng(7)
    n = 3000
    xyz = (rng.random((n, 3)) * np.array([9.0, 7.0, 11.0])).astype(np.float32)
    t = rng.integers(0, 3, n).astype(np.uint8)
    d = (rng.random(n) * 3.0).astype(np.float32)
    org = xyz.min(axis=0)
    dims = tuple(int(np.floor((xyz[:, a].max() - org[a]) / h)) + 1 for a in range(3))
    info = dict(dims=dims, origin=tuple(float(v) for v in org), cell=h, n_cells=dims[0] * dims[1] * dims[2])
    got = bench.candidate_tests(torch.from_numpy(xyz), torch.from_numpy(t), torch.from_numpy(d), [1], [1, 2], 1.0,
                                info, stencil, cell_scale=cs)
    inv_h = np.float32(1.0 / h)
    cn = _cells_np(xyz[np.isin(t, [1, 2])], org, inv_h, dims)
    cc = _cells_np(xyz[(t == 1) & (d >= 1.0)], org, inv_h, dims)
    want = sum(int(((np.abs(cn - c).max(axis=1) <= stencil) & _kept(cn - c, cs)).sum()) for c in cc)
    assert got == want > 0
    if cs is not None and cs < 1 / stencil + 0.1:
        assert got < sum(int((np.abs(cn - c).max(axis=1) <= stencil).sum()) for c in cc) or stencil == 2


def test_stored_traffic_guard():
    cfg = {"all-all": {"cell_scale": 0.5, "dense_min": 0, "split": 1}, "Sc-Sc": {"cell_scale": 0.5, "dense_min": 0, "split": 0}}
    v = bench.stored_traffic("needle2g", cfg)
    # either the stored figures (sources unchanged since the capture) or None; never for another setup
    assert v is None or (v["combination"] == "all-all" and v["kernels"]["rdf_sym"] > 0)
    assert bench.stored_traffic("needle2g", {**cfg, "Sc-Sc": {"cell_scale": 1.0, "dense_min": 0, "split": 0}}) is None
    assert bench.stored_traffic("cylinder200k", cfg) is None


def _combo(name, split, near, sym, n_pairs):
    by = {"query": near, "rdf_sym": sym} if split else {"query": near}
    return dict(name=name, n_nbr=1000, n_cells=100, n_central=900, n_ctr_typed=950, n_pairs_local=n_pairs,
                subset=True, candidates=near + sym, candidates_by_pass=by, split=split)


def test_rooflines_dominant_kernel_and_traffic():
    """The roofline names the query family with the most time; its traffic is reported per launch
    only when every launch of that family belongs to the recorded combination."""
    peaks = {"fp32_scalar_gops": 40000.0, "fp32_packed_gops": 40000.0, "smem_atomic_gops": 10000.0,
             "num_sms": 152, "sm_mhz": 2070.0}
    st = {"n_ions": 1000, "combos": [_combo("all-all", True, 4e9, 1e10, 5e8), _combo("Sc-Sc", False, 1e8, 0, 1e6)]}
    zero = (0, 0.0)
    prof = {f: zero for f in bench.FAMS}
    prof.update(query=(4, 100.0), knn_full=(2, 4.0), rdf_sym=(2, 300.0), scan=(4, 10.0))
    traffic = {"combination": "all-all", "kernels": {"query": 5e9, "knn_full": 1e8, "rdf_sym": 2e10}}
    r = bench.rooflines(prof, st, 2, peaks, 6000.0, "measured", traffic)
    assert r["family"] == "rdf_sym" and r["traffic"] == 2e10
    sym_tf = 9 * 1e10 * 2 / 0.3 / 1e12
    assert abs(r["achieved"] - sym_tf) < 1e-9 and abs(r["frac"] - sym_tf / 40.0) < 1e-9
    # k_query_warp also runs for Sc-Sc: no per-launch traffic for that family, the record kept beside it
    assert r["by_kernel"]["query"]["traffic"] is None and r["by_kernel"]["query"]["traffic_recorded"] == 5e9
    assert r["by_kernel"]["knn_full"]["achieved_tflops"] is None
    allq = 9 * (4e9 + 1e10 + 1e8) * 2 / 0.404 / 1e12
    assert abs(r["all_query_passes"]["achieved"] - allq) < 1e-6
    assert bench.rooflines(prof, st, 2, peaks, 6000.0, "measured", None)["traffic"] is None


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


@pytest.mark.parametrize("stencil,h,cs", [(2, 1.0, 0.5), (3, 0.7, 1 / 3)])
def test_symmetric_pass_test_count_brute_force(stencil, h, cs):
    """The symmetric RDF pass tests every unordered pair of records whose cells are within the
    searched stencil once: (sum over records of their stencil population - n) / 2, by brute force."""
    rng = np.random.default_rng(8)
    n = 2500
    xyz = (rng.random((n, 3)) * np.array([6.0, 5.0, 7.0])).astype(np.float32)
    t = rng.integers(0, 2, n).astype(np.uint8)
    d = np.full(n, np.nan, np.float32)  # no d_srf filter applies to the record count
    org = xyz.min(axis=0)
    dims = tuple(int(np.floor((xyz[:, a].max() - org[a]) / h)) + 1 for a in range(3))
    info = dict(dims=dims, origin=tuple(float(v) for v in org), cell=h, n_cells=dims[0] * dims[1] * dims[2])
    full = bench.candidate_tests(torch.from_numpy(xyz), torch.from_numpy(t), torch.from_numpy(d), "all", "all", 0.0,
                                 info, stencil, all_records=True, cell_scale=cs)
    c = _cells_np(xyz, org, np.float32(1.0 / h), dims)
    dc = c[:, None, :] - c[None, :, :]
    near = (np.abs(dc).max(axis=2) <= stencil) & _kept(dc, cs)
    pairs = int(np.triu(near, k=1).sum())
    assert (full - n) // 2 == pairs and (full - n) % 2 == 0


def test_octant_tests_brute_force():
    """The near kNN pass tests every central against the records of its own 2 x 2 x 2 block:
    its cell and the neighbour on the side of its half along each axis (clipped at the faces)."""
    rng = np.random.default_rng(9)
    n = 3000
    xyz = (rng.random((n, 3)) * np.array([7.0, 5.0, 9.0])).astype(np.float32)
    t = rng.integers(0, 3, n).astype(np.uint8)
    d = (rng.random(n) * 3.0).astype(np.float32)
    h = 1.0
    org = xyz.min(axis=0)
    dims = tuple(int(np.floor((xyz[:, a].max() - org[a]) / h)) + 1 for a in range(3))
    info = dict(dims=dims, origin=tuple(float(v) for v in org), cell=h, n_cells=dims[0] * dims[1] * dims[2])
    got = bench.octant_tests(torch.from_numpy(xyz), torch.from_numpy(t), torch.from_numpy(d), [1], [0, 1], 1.0, info)
    inv_h = np.float32(1.0 / h)
    cn = _cells_np(xyz[np.isin(t, [0, 1])], org, inv_h, dims)
    P = xyz[(t == 1) & (d >= 1.0)]
    u = (P - org.astype(np.float32)).astype(np.float32) * inv_h
    cc = np.clip(np.floor(u).astype(np.int64), 0, np.array(dims) - 1)
    side = np.where(u - cc.astype(np.float32) >= 0.5, 1, -1)
    want = 0
    for c, sg in zip(cc, side):
        lo, hi = np.minimum(c, c + sg), np.maximum(c, c + sg)
        want += int(np.all((cn >= lo) & (cn <= hi), axis=1).sum())
    assert got == want > 0


def test_row_widths_rule():
    """Half-size cells keep every cell of the 5 x 5 x 5 stencil; third-size cells drop the 4 far
    corner cells of each octant (32 of 343); cells of 0.75 r_cut drop the rows (+-2, +-2) and the
    ends of the rows with one offset of 2."""
    assert bench.row_widths(2, 0.5) == [[2] * 5] * 5
    w3 = bench.row_widths(3, 1 / 3)
    assert sum(2 * w + 1 for row in w3 for w in row if w >= 0) == 343 - 32
    assert w3[0][0] == 1 and w3[0][1] == 2 and w3[0][2] == 3 and w3[3][3] == 3
    w = bench.row_widths(2, 0.75)
    assert w[0][0] == -1 and w[4][4] == -1 and w[0][2] == 1 and w[1][0] == 1 and w[2][2] == 2
