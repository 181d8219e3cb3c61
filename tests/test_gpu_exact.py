"""GPU parity of the exact kNN / RDF path against the oracle (bit-exact integers).

Every case calls the CUDA library through its C ABI (via the thin binding)
and the oracle on the same seeded inputs, and compares every histogram bin,
every counter and, where requested, every per-central output.
"""
import math

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


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def run_gpu(ps, xyz, t, d, ctr, nbr, dmin, bins, ks, per_central=False, r_cut=None, cell_scale=1.0, rdf=True,
            dense_min=0, split=False):
    X, T, D = _dev(xyz, t, d)
    r0, dr, nb = bins
    rc = r_cut if r_cut is not None else float(np.float32(r0 + nb * dr)) * (1 + 1e-6)
    g = ps.Grid(X.shape[0], cell_scale, dense_min, split).build(X, T, nbr, rc)
    out = ps.spatstat(g, D, ctr, dmin, bins, ks, rdf=rdf, per_central=per_central)
    torch.cuda.synchronize()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    g.close()
    return res


def assert_same(gpu, ref, ks, per_central=False, rdf=True):
    meta = gpu["meta"].astype(np.uint64)
    assert meta[3] == 0, f"device status {meta[3]}"
    assert meta[0] == ref["n_central"]
    if rdf:
        np.testing.assert_array_equal(gpu["rdf"].astype(np.uint64), ref["rdf"])
        assert meta[1] == ref["n_pairs"] and meta[2] == ref["rdf_below"]
    if ks:
        np.testing.assert_array_equal(gpu["knn"].astype(np.uint64), ref["knn"])
        np.testing.assert_array_equal(meta[4::2], ref["not_found"])
        np.testing.assert_array_equal(meta[5::2], ref["knn_below"])
    if per_central:
        if per_central != "kth":
            np.testing.assert_array_equal(gpu["n_within"].astype(np.uint32), ref["n_within"])
        if ks:
            a, b = gpu["kth_d2"], ref["kth_d2"]
            both_nan = np.isnan(a) & np.isnan(b)
            np.testing.assert_array_equal(np.where(both_nan, 0, a), np.where(both_nan, 0, b))


CASES = [
    ("all", "all", 0.0, [1, 2, 7, 32]),
    ([1], [1], 1.0, [1, 3]),
    ([0], [1, 2], 0.5, [1, 5, 10]),
    ([2], "all", -1.0, [4]),
    ([0, 1], [0], 0.8, []),
]


@pytest.mark.parametrize("n,L,seed", [(3000, 5.0, 101), (20000, 9.0, 102), (777, 3.1, 103)])
def test_poisson_cube_all_masks(ps, orc, spec, n, L, seed):
    xyz, t, d = spec.cube(seed, n, L, (0.6, 0.3, 0.1))
    bins = (0.0, 0.02, 75)
    for ctr, nbr, dmin, ks in CASES:
        g = run_gpu(ps, xyz, t, d, ctr, nbr, dmin, bins, ks, per_central=True)
        r = orc.spatstat(xyz, t, d, ctr, nbr, dmin, *bins, ks, per_central=True)
        assert_same(g, r, ks, per_central=True)


def test_cylinder_200k_all_all_full_size(ps, orc, spec):
    """The 200,000-ion Poisson cylinder: all-all, d_srf >= 1, k = 1, RDF on [0, 0.01, 2]."""
    xyz, t, d = spec.cylinder_small()
    bins = ps.bins_from_spec(0.0, 0.01, 2.0)
    g = run_gpu(ps, xyz, t, d, "all", "all", 1.0, bins, [1], per_central=True)
    r = orc.spatstat(xyz, t, d, "all", "all", 1.0, *bins, [1], per_central=True)
    assert 140000 < r["n_central"] < 142500
    assert_same(g, r, [1], per_central=True)


@pytest.mark.parametrize("ctr,nbr", [([1], [1]), ([0], [1]), ([2], [2]), ([1], [0, 2])])
def test_cylinder_200k_type_pairs(ps, orc, spec, ctr, nbr):
    xyz, t, d = spec.cylinder_small()
    bins = ps.bins_from_spec(0.0, 0.01, 2.0)
    ks = [1, 5, 10]
    g = run_gpu(ps, xyz, t, d, ctr, nbr, 1.0, bins, ks)
    r = orc.spatstat(xyz, t, d, ctr, nbr, 1.0, *bins, ks)
    assert_same(g, r, ks)


def test_needle_8m_sc_sc_si_si_full_size(ps, orc, spec):
    """The ~8e6-ion needle: Sc-Sc and Si-Si, k in {1, 5, 10}, r = [0, 0.01, 2], d_srf >= 2."""
    xyz, t, d = spec.needle(spec.needle_8m_params())
    bins = ps.bins_from_spec(0.0, 0.01, 2.0)
    ks = [1, 5, 10]
    for typ in (1, 2):
        g = run_gpu(ps, xyz, t, d, [typ], [typ], 2.0, bins, ks, per_central=True)
        r = orc.spatstat(xyz, t, d, [typ], [typ], 2.0, *bins, ks, per_central=True)
        assert r["n_central"] > 1000
        assert_same(g, r, ks, per_central=True)


def test_simple_cubic_lattice_exact_shells(ps, orc, spec):
    xyz, t, d = spec.simple_cubic(24, 0.25, 0.125)
    bins = (0.0, 0.01, 200)
    ks = list(range(1, 33))
    g = run_gpu(ps, xyz, t, d, "all", "all", 2.0, bins, ks, per_central=True)
    r = orc.spatstat(xyz, t, d, "all", "all", 2.0, *bins, ks, per_central=True)
    assert_same(g, r, ks, per_central=True)
    assert g["rdf"][25] == 512 * 6 and g["rdf"][24] == 0 and g["rdf"][50] == 512 * 6


def test_duplicates_edges_and_below_range(ps, orc):
    rng = np.random.default_rng(9)
    base = rng.uniform(0, 3, (400, 3)).astype(np.float32)
    xyz = np.concatenate([base, base[:50], base[:10] + np.float32(0.25)]).astype(np.float32)
    t = np.zeros(xyz.shape[0], np.uint8)
    d = np.full(xyz.shape[0], 5.0, np.float32)
    for bins in [(0.0, 0.01, 150), (0.3, 0.01, 90), (0.25, 0.05, 10)]:
        ks = [1, 2, 3, 9]
        g = run_gpu(ps, xyz, t, d, "all", "all", 0.0, bins, ks, per_central=True)
        r = orc.spatstat(xyz, t, d, "all", "all", 0.0, *bins, ks, per_central=True)
        assert_same(g, r, ks, per_central=True)
    assert r["rdf_below"] > 0 and r["knn_below"].sum() > 0


def test_dense_cells_many_chunks_and_batches(ps, orc, spec):
    # 120 ions/nm^3: ~1000 centrals per cell and ~26k candidates per cell (several staged chunks)
    xyz, t, d = spec.cube(104, 20000, (20000 / 120.0) ** (1 / 3), (0.5, 0.5))
    bins = (0.0, 0.02, 100)
    ks = [1, 16]
    r = orc.spatstat(xyz, t, d, "all", "all", 0.0, *bins, ks, per_central=True)
    for dense_min in (0, 64):
        g = run_gpu(ps, xyz, t, d, "all", "all", 0.0, bins, ks, per_central=True, dense_min=dense_min)
        assert_same(g, r, ks, per_central=True)


def test_extreme_clusters_split_lanes(ps, orc, spec):
    """Two dense blobs in a sparse cloud: the blobs' cells hold 16-32x and > 32x the cloud's mean
    stencil population, so their centrals are tested by 2 and 4 lanes each (partial top-k lists
    merged by shuffles)."""
    rng = np.random.default_rng(77)
    bg = (rng.random((8000, 3)) * 40.0).astype(np.float32)
    a = (np.array([12.0, 20.0, 20.0]) + rng.normal(0, 0.25, (6000, 3))).astype(np.float32)
    b = (np.array([28.0, 20.0, 20.0]) + rng.normal(0, 0.25, (1300, 3))).astype(np.float32)
    xyz = np.concatenate([bg, a, b])
    t = rng.integers(0, 2, xyz.shape[0]).astype(np.uint8)
    d = np.full(xyz.shape[0], 5.0, np.float32)
    bins = (0.0, 0.01, 200)
    X, T = _dev(xyz, t)
    g = ps.Grid(xyz.shape[0]).build(X, T, "all", 2.0 * (1 + 1e-6))
    info = g.info()
    g.close()
    mean_stencil = 27.0 * info["n_nbr"] / info["n_cells"]
    assert 16 * mean_stencil < 1300 < 32 * mean_stencil and 6000 > 32 * mean_stencil
    for ctr, nbr, ks in (("all", "all", [1, 5, 12]), ([1], "all", [3, 32]), ("all", [0], [7])):
        gg = run_gpu(ps, xyz, t, d, ctr, nbr, 0.0, bins, ks, per_central=True)
        r = orc.spatstat(xyz, t, d, ctr, nbr, 0.0, *bins, ks, per_central=True)
        assert_same(gg, r, ks, per_central=True)


@pytest.mark.parametrize("cell_scale,dense_min", [(1.0, 0), (1.0, 40), (0.5, 0), (0.5, 8), (0.7, 0), (0.75, 0),
                                                  (0.75, 8), (1.3, 1), (1 / 3, 0), (1 / 3, 4), (0.4, 0)])
def test_kernel_variants_stencils(ps, orc, spec, cell_scale, dense_min):
    """27-, 125- and 343-cell stencils (the last two less the cells that cannot hold a pair
    within r_cut: the 8 corners at cell_scale 0.7, whole rows at 0.75, the 32 far corners at 1/3),
    warp kernel alone (49 stencil rows in two run-table rounds at 1/3) and with the CTA kernel
    taking the dense cells."""
    xyz, t, d = spec.cube(111, 12000, 7.5, (0.7, 0.2, 0.1))
    bins = (0.0, 0.02, 80)
    for ctr, nbr, dmin, ks in [("all", "all", 0.5, [1, 3, 12]), ([1], [1, 2], 0.0, [2]), ([0], "all", 1.0, [32])]:
        g = run_gpu(ps, xyz, t, d, ctr, nbr, dmin, bins, ks, per_central=True, cell_scale=cell_scale,
                    dense_min=dense_min)
        r = orc.spatstat(xyz, t, d, ctr, nbr, dmin, *bins, ks, per_central=True)
        assert_same(g, r, ks, per_central=True)


def test_coarse_cells_cell_scale(ps, orc, spec):
    xyz, t, d = spec.cube(105, 5000, 6.0, (0.5, 0.5))
    bins = (0.0, 0.02, 60)
    g = run_gpu(ps, xyz, t, d, "all", [1], 0.5, bins, [3], cell_scale=1.7)
    r = orc.spatstat(xyz, t, d, "all", [1], 0.5, *bins, [3])
    assert_same(g, r, [3])


def test_empty_sets(ps, orc, spec):
    xyz, t, d = spec.cube(106, 2000, 4.0, (1.0,))
    bins = (0.0, 0.02, 50)
    # no neighbours of type 7: every central is "not found"
    g = run_gpu(ps, xyz, t, d, "all", [7], 0.0, bins, [1, 2])
    r = orc.spatstat(xyz, t, d, "all", [7], 0.0, *bins, [1, 2])
    assert_same(g, r, [1, 2])
    assert g["meta"][4] == 2000
    # no centrals
    g = run_gpu(ps, xyz, t, d, [3], "all", 0.0, bins, [1])
    assert g["meta"][0] == 0 and g["rdf"].sum() == 0 and g["knn"].sum() == 0
    # d_srf threshold above every ion
    g = run_gpu(ps, xyz, t, d, "all", "all", 100.0, bins, [1])
    assert g["meta"][0] == 0


def test_single_ion_and_empty_cloud(ps):
    xyz = np.array([[1.0, 2.0, 3.0]], np.float32)
    g = run_gpu(ps, xyz, np.zeros(1, np.uint8), np.ones(1, np.float32), "all", "all", 0.0, (0.0, 0.1, 10), [1])
    assert g["meta"][0] == 1 and g["meta"][4] == 1 and g["rdf"].sum() == 0
    X = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    T = torch.zeros(0, dtype=torch.uint8, device="cuda")
    grid = ps.Grid(16).build(X, T, "all", 1.0)
    out = ps.spatstat(grid, None, "all", 0.0, (0.0, 0.1, 10), [1])
    assert int(out["meta"][0]) == 0 and int(out["rdf"].sum()) == 0
    grid.close()


def test_repeated_queries_overwrite_and_streams(ps, orc, spec):
    xyz, t, d = spec.cube(107, 6000, 6.0, (0.7, 0.3))
    X, T, D = _dev(xyz, t, d)
    bins = (0.0, 0.02, 80)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g = ps.Grid(X.shape[0]).build(X, T, "all", 1.61, stream=s)
        outs = [ps.spatstat(g, D, [1], 0.5, bins, [2], stream=s, check=False) for _ in range(3)]
    s.synchronize()
    r = orc.spatstat(xyz, t, d, [1], "all", 0.5, *bins, [2])
    for o in outs:
        assert_same({k: v.cpu().numpy() for k, v in o.items() if v is not None}, r, [2])
    info = g.info()
    assert info["n_nbr"] == 6000 and info["cell"] >= 1.61 and info["status"] == 0
    g.close()


def test_single_k_and_rdf_entry_points(ps, orc, spec):
    xyz, t, d = spec.cube(108, 4000, 5.5, (0.5, 0.5))
    X, T, D = _dev(xyz, t, d)
    bins = (0.0, 0.02, 70)
    g = ps.Grid(X.shape[0]).build(X, T, [0], 1.4000001)
    h, meta = ps.knn_hist(g, D, [1], 0.3, 6, bins)
    hr, metar = ps.rdf_hist(g, D, [1], 0.3, bins)
    r = orc.spatstat(xyz, t, d, [1], [0], 0.3, *bins, [6])
    np.testing.assert_array_equal(h.cpu().numpy().astype(np.uint64), r["knn"][0])
    np.testing.assert_array_equal(hr.cpu().numpy().astype(np.uint64), r["rdf"])
    assert int(meta[4]) == r["not_found"][0] and int(metar[0]) == r["n_central"]
    g.close()


def test_non_finite_input_reports_status(ps, spec):
    xyz, t, d = spec.cube(109, 1000, 4.0, (1.0,))
    xyz[17, 1] = np.nan
    xyz[33, 0] = np.inf
    X, T, D = _dev(xyz, t, d)
    g = ps.Grid(X.shape[0]).build(X, T, "all", 1.0)
    assert g.info()["status"] == 2
    with pytest.raises(ps.PSError) as e:
        ps.spatstat(g, D, "all", 0.0, (0.0, 0.1, 10), [1])
    assert e.value.code == 2
    g.close()


def test_host_argument_errors(ps, spec):
    xyz, t, d = spec.cube(110, 500, 3.0, (1.0,))
    X, T, D = _dev(xyz, t, d)
    g = ps.Grid(X.shape[0]).build(X, T, "all", 1.0)
    with pytest.raises(ps.PSError) as e:
        ps.spatstat(g, D, "all", 0.0, (0.0, 0.1, 11), [1])  # stop 1.1 > r_cut 1.0
    assert e.value.code == 1
    for ks in ([0], [33]):
        with pytest.raises(ps.PSError) as e:
            ps.spatstat(g, D, "all", 0.0, (0.0, 0.1, 10), ks)
        assert e.value.code == 6
    with pytest.raises(ps.PSError) as e:
        ps.spatstat(g, D, "all", 0.0, (0.0, 0.0001, 9000), [1])
    assert e.value.code == 6
    g2 = ps.Grid(100)
    with pytest.raises(ps.PSError) as e:
        g2.build(X, T, "all", 1.0)
    assert e.value.code == 7
    g.close()
    g2.close()
