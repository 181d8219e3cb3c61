"""GPU parity of maximum-separation clustering (ps_cluster) against the oracle: every label,
both size histograms and every counter, bit-exact; on a chain at exactly d_max, lattices,
precipitate needles (Sc) over a d_max sweep, random blobs, the grid options, empty sets and
argument checks."""
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


def _gpu(ps, xyz, t, d, types, d_max, n_min, dsrf_min=0.0, hist_len=1024, cell_scale=1.0, r_cut=None):
    X, T, D = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (xyz, t, d))
    g = ps.Grid(X.shape[0], cell_scale).build(X, T, types, r_cut or d_max * (1 + 1e-6))
    o = ps.cluster(g, D, d_max, n_min, dsrf_min, hist_len)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in o.items()}
    g.close()
    return res


def _same(ps, orc, xyz, t, d, types, d_max, n_min, dsrf_min=0.0, hist_len=1024, **kw):
    g = _gpu(ps, xyz, t, d, types, d_max, n_min, dsrf_min, hist_len, **kw)
    r = orc.cluster(xyz, t, d, types, d_max, n_min, dsrf_min, hist_len)
    assert g["meta"][4] == 0
    np.testing.assert_array_equal(g["label"].astype(np.uint32), r["label"])
    np.testing.assert_array_equal(g["size_hist"].astype(np.uint64), r["size_hist"])
    np.testing.assert_array_equal(g["interior_hist"].astype(np.uint64), r["interior_hist"])
    assert tuple(int(v) for v in g["meta"][:4]) == (r["n_set"], r["n_clusters"], r["n_clustered"], r["n_interior"])
    return r


def test_chain_at_exactly_d_max(ps, orc):
    n = 300
    xyz = np.zeros((n, 3), np.float32)
    xyz[:, 0] = np.arange(n, dtype=np.float32) * np.float32(0.5)
    t = np.ones(n, np.uint8)
    d = np.full(n, 5.0, np.float32)
    r = _same(ps, orc, xyz, t, d, [1], 0.5, 2)
    assert r["n_clusters"] == 1
    r = _same(ps, orc, xyz, t, d, [1], 0.4999, 1, r_cut=0.5)
    assert r["n_clusters"] == n


def test_lattice(ps, orc, spec):
    xyz, t, d = spec.simple_cubic(20)
    _same(ps, orc, xyz, t, d, [0], 0.25, 5)
    _same(ps, orc, xyz, t, d, [0], 0.24, 1, r_cut=0.25)


@pytest.mark.parametrize("d_max", [0.10, 0.30, 0.50, 0.70])
def test_needle_sc_sweep(ps, orc, spec, d_max):
    xyz, t, d = spec.needle(spec.needle_params(r_top=10.0, half_angle_deg=10.0, height=30.0, seed=12))
    r = _same(ps, orc, xyz, t, d, [1], d_max, 5, dsrf_min=1.0, hist_len=512)
    if d_max >= 0.5:
        assert r["n_clusters"] > 0


@pytest.mark.parametrize("seed", [1, 2])
def test_random_blobs_and_options(ps, orc, seed):
    rng = np.random.default_rng(seed)
    n = 30000
    xyz = (rng.random((n, 3)) * 12.0).astype(np.float32)
    for c in rng.random((25, 3)) * 12.0:
        k = int(rng.integers(50, 400))
        xyz[rng.choice(n, k, replace=False)] = (c + rng.normal(0, 0.3, (k, 3))).astype(np.float32)
    t = rng.integers(0, 3, n).astype(np.uint8)
    d = (rng.random(n) * 3.0).astype(np.float32)
    for types, d_max, n_min, cs in (([1, 2], 0.3, 3, 1.0), ("all", 0.25, 10, 0.5), ([0], 0.4, 2, 0.75)):
        _same(ps, orc, xyz, t, d, types, d_max, n_min, 1.0, 64, cell_scale=cs)


def test_empty_and_single(ps, orc, spec):
    xyz, t, d = spec.cylinder(3, 2000, 3.0, 3.0, (1.0,))
    r = _same(ps, orc, xyz, t, d, [7], 0.5, 1)
    assert r["n_set"] == 0 and r["n_clusters"] == 0
    _same(ps, orc, xyz[:1], t[:1], d[:1], "all", 0.5, 1)


def test_argument_checks(ps, spec):
    xyz, t, d = spec.cylinder(4, 1000, 3.0, 3.0, (1.0,))
    X, T, D = (torch.from_numpy(a).cuda() for a in (xyz, t, d))
    g = ps.Grid(1000).build(X, T, "all", 0.5)
    with pytest.raises(RuntimeError):
        ps.cluster(g, D, 0.6, 2)  # d_max above r_cut
    with pytest.raises(RuntimeError):
        ps.cluster(g, D, 0.4, 0)
    with pytest.raises(RuntimeError):
        ps.cluster(g, D, 0.4, 2, hist_len=1)
    g.close()
