"""GPU parity of the exact query in passes (ps_grid_opts.split) against the oracle, bit for bit.

With half-size cells, central types among the neighbour types and the RDF requested, the query
runs as (1) kNN within the cell edge on 27 cells, (2) the full-radius kNN of the centrals that
have fewer than k neighbours there, (3) the RDF over unordered pairs, each tested once and
counted once per central end.  Every histogram bin, counter and per-central k-th distance
must equal the oracle's -- including clouds where most centrals need the full search (sparse
types), cells of more than 32 records (several lane chunks), duplicates and exact edges,
r0 > 0 (pairs below the first edge) and the cases that keep the one-pass query (n_within
requested, central types outside the neighbour set, full-size cells)."""
import numpy as np
import pytest

from test_gpu_exact import _dev, assert_same, run_gpu

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


CASES = [
    ("all", "all", 0.0, [1, 2, 7, 32]),
    ([1], [1], 1.0, [1, 3]),
    ([1], [0, 1], 0.5, [1, 5, 10]),
    ("all", "all", 1.0, []),
    ([0, 1], [0, 1, 2], -1.0, [12]),
    ([0], [1, 2], 0.5, [1, 5]),  # central types outside the neighbour set: one pass
]


@pytest.mark.parametrize("n,L,seed", [(3000, 5.0, 201), (20000, 9.0, 202), (777, 3.1, 203)])
def test_poisson_cube_split(ps, orc, spec, n, L, seed):
    xyz, t, d = spec.cube(seed, n, L, (0.6, 0.3, 0.1))
    bins = (0.0, 0.02, 75)
    for ctr, nbr, dmin, ks in CASES:
        for cs in (0.5, 0.75, 1 / 3):
            g = run_gpu(ps, xyz, t, d, ctr, nbr, dmin, bins, ks, per_central="kth", cell_scale=cs, split=True)
            r = orc.spatstat(xyz, t, d, ctr, nbr, dmin, *bins, ks, per_central=True)
            assert_same(g, r, ks, per_central="kth")


def test_cylinder_200k_split_full_size(ps, orc, spec):
    xyz, t, d = spec.cylinder_small()
    bins = ps.bins_from_spec(0.0, 0.01, 2.0)
    r = orc.spatstat(xyz, t, d, "all", "all", 1.0, *bins, [1, 10], per_central=True)
    g = run_gpu(ps, xyz, t, d, "all", "all", 1.0, bins, [1, 10], per_central="kth", cell_scale=0.5, split=True)
    assert_same(g, r, [1, 10], per_central="kth")
    # n_within requested: the one-pass query, same histograms
    g = run_gpu(ps, xyz, t, d, "all", "all", 1.0, bins, [1, 10], per_central=True, cell_scale=0.5, split=True)
    assert_same(g, r, [1, 10], per_central=True)


def test_cylinder_200k_benchmark_configuration(ps, orc, spec):
    """The 2e5 cylinder as the benchmark runs it (all-all, k = 1, r = [0, 0.01, 2] nm, d_srf >= 1
    nm) in the configuration its autotuner picks there: third-size cells, the query in passes."""
    xyz, t, d = spec.cylinder_small()
    bins = ps.bins_from_spec(0.0, 0.01, 2.0)
    r = orc.spatstat(xyz, t, d, "all", "all", 1.0, *bins, [1], per_central=True)
    g = run_gpu(ps, xyz, t, d, "all", "all", 1.0, bins, [1], per_central="kth", cell_scale=1 / 3, split=True)
    assert_same(g, r, [1], per_central="kth")


@pytest.mark.parametrize("cell_scale", [0.5, 1 / 3])
def test_needle_8m_sparse_types_split(ps, orc, spec, cell_scale):
    """Sc-Sc: almost no Sc has 5 Sc neighbours within 1 nm (0.67 nm with third-size cells), so
    nearly every central takes the full-radius fallback (49 stencil rows with third-size cells)."""
    xyz, t, d = spec.needle(spec.needle_8m_params())
    bins = ps.bins_from_spec(0.0, 0.01, 2.0)
    for ctr, nbr, ks in (([1], [1], [1, 5, 10]), ([2], [2], [1, 5, 10]), ([1], [1, 2], [2])):
        g = run_gpu(ps, xyz, t, d, ctr, nbr, 2.0, bins, ks, per_central="kth", cell_scale=cell_scale, split=True)
        r = orc.spatstat(xyz, t, d, ctr, nbr, 2.0, *bins, ks, per_central=True)
        assert_same(g, r, ks, per_central="kth")


def test_lattice_duplicates_edges_split(ps, orc, spec):
    xyz, t, d = spec.simple_cubic(24, 0.25, 0.125)
    ks = list(range(1, 33))
    g = run_gpu(ps, xyz, t, d, "all", "all", 2.0, (0.0, 0.01, 200), ks, per_central="kth", cell_scale=0.5,
                split=True)
    r = orc.spatstat(xyz, t, d, "all", "all", 2.0, 0.0, 0.01, 200, ks, per_central=True)
    assert_same(g, r, ks, per_central="kth")
    rng = np.random.default_rng(19)
    base = rng.uniform(0, 3, (400, 3)).astype(np.float32)
    xyz = np.concatenate([base, base[:50], base[:10] + np.float32(0.25)]).astype(np.float32)
    t = (np.arange(xyz.shape[0]) % 3 == 0).astype(np.uint8)
    d = rng.uniform(0, 1, xyz.shape[0]).astype(np.float32)
    for bins in [(0.0, 0.01, 150), (0.3, 0.01, 90), (0.25, 0.05, 10)]:
        for ctr, dmin in (("all", 0.0), ("all", 0.5), ([1], 0.2)):
            ks = [1, 2, 3, 9]
            g = run_gpu(ps, xyz, t, d, ctr, "all", dmin, bins, ks, per_central="kth", cell_scale=0.5, split=True)
            r = orc.spatstat(xyz, t, d, ctr, "all", dmin, *bins, ks, per_central=True)
            assert_same(g, r, ks, per_central="kth")


def test_dense_cells_many_lane_chunks_split(ps, orc, spec):
    # 120 ions/nm^3 with cells of ~1 nm: ~120 records per cell, four chunks of 32 lanes
    xyz, t, d = spec.cube(204, 20000, (20000 / 120.0) ** (1 / 3), (0.5, 0.5))
    bins = (0.0, 0.02, 100)
    for ctr, nbr, ks in (("all", "all", [1, 16]), ([1], "all", [3]), ([0], [0], [])):
        r = orc.spatstat(xyz, t, d, ctr, nbr, 0.3, *bins, ks, per_central=True)
        g = run_gpu(ps, xyz, t, d, ctr, nbr, 0.3, bins, ks, per_central="kth", cell_scale=0.5, split=True)
        assert_same(g, r, ks, per_central="kth")


def test_split_edge_cases(ps, orc, spec):
    xyz, t, d = spec.cube(206, 2000, 4.0, (1.0,))
    bins = (0.0, 0.02, 50)
    for ctr, dmin, ks in (([3], 0.0, [1]), ("all", 100.0, [1]), ("all", 0.0, [1, 2])):
        g = run_gpu(ps, xyz, t, d, ctr, "all", dmin, bins, ks, cell_scale=0.5, split=True)
        r = orc.spatstat(xyz, t, d, ctr, "all", dmin, *bins, ks)
        assert_same(g, r, ks)
    one = np.array([[1.0, 2.0, 3.0]], np.float32)
    g = run_gpu(ps, one, np.zeros(1, np.uint8), np.ones(1, np.float32), "all", "all", 0.0, (0.0, 0.1, 10), [1],
                cell_scale=0.5, split=True)
    assert g["meta"][0] == 1 and g["meta"][4] == 1 and g["rdf"].sum() == 0
    # repeated queries on one grid, with and without the kNN part
    X, T, D = _dev(xyz, t, d)
    grid = ps.Grid(X.shape[0], 0.5, 0, True).build(X, T, "all", 1.0 * (1 + 1e-6))
    for ks in ([4], [], [1, 8], [4]):
        o = ps.spatstat(grid, D, "all", 0.2, bins, ks)
        r = orc.spatstat(xyz, t, d, "all", "all", 0.2, *bins, ks)
        assert_same({k: v.cpu().numpy() for k, v in o.items() if v is not None}, r, ks)
    grid.close()


@pytest.mark.parametrize("bins", [(0.0, 0.01, 200), (0.0, 0.001, 2000), (0.5, 0.005, 300), (0.0, 0.25, 8),
                                  (0.0, 2.0, 1)])
def test_bin_lookup_regimes(ps, orc, spec, bins):
    """The bin of a pair comes from a lookup table on the float32 bit pattern of d2 where the
    edges are far enough apart (one interior edge per table cell), else from an approximate
    square root checked against the edges: fine bins (no table), r0 > 0, a few wide bins and a
    single bin, in both query forms."""
    xyz, t, d = spec.cube(207, 6000, 6.0, (0.7, 0.3))
    r = orc.spatstat(xyz, t, d, "all", "all", 0.5, *bins, [1, 4], per_central=True)
    for split in (False, True):
        g = run_gpu(ps, xyz, t, d, "all", "all", 0.5, bins, [1, 4], per_central="kth", cell_scale=0.5, split=split)
        assert_same(g, r, [1, 4], per_central="kth")


@pytest.mark.parametrize("rho,cs", [(3.0, 0.5), (12.0, 0.5), (33.0, 0.5), (33.0, 1 / 3), (120.0, 1 / 3)])
def test_split_lane_chunks(ps, orc, spec, rho, cs):
    """Cells of few and of many records: 3, 12 and 33 ions per nm^3 on cells of ~1 nm^3 (items
    of 8, 4, 2 and 1 lanes per central in the near pass, record groups of every size in the
    symmetric pass), and third-size cells (~0.3 nm^3) at 33 and 120 ions per nm^3."""
    L = 9.0
    xyz, t, d = spec.cube(208, int(rho * L**3), L, (0.6, 0.4))
    bins = (0.0, 0.02, 100)
    for ctr, nbr, ks in (("all", "all", [1, 6]), ([1], [0, 1], [2]), ([0], [0], [])):
        r = orc.spatstat(xyz, t, d, ctr, nbr, 0.7, *bins, ks, per_central=True)
        g = run_gpu(ps, xyz, t, d, ctr, nbr, 0.7, bins, ks, per_central="kth", cell_scale=cs, split=True)
        assert_same(g, r, ks, per_central="kth")
