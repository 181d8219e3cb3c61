"""Pins for the maximum-separation clustering oracle:

* the closed link rule d <= d_max on points spaced exactly d_max apart (float32-exact spacing);
* simple-cubic lattices, where the components follow from the spacing alone;
* an independent brute force (numpy pair test + scipy connected components) on random clouds;
* invariance of the partition under a permutation of the input order; the type mask.
"""
import numpy as np
import pytest

scipy_sparse = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def test_chain_closed_link_rule(orc):
    n = 40
    xyz = np.zeros((n, 3), np.float32)
    xyz[:, 0] = np.arange(n, dtype=np.float32) * np.float32(0.5)
    t = np.ones(n, np.uint8)
    d = np.full(n, 5.0, np.float32)
    r = orc.cluster(xyz, t, d, [1], 0.5, 2)  # (0.5)^2 = 0.25 exactly: neighbours at exactly d_max link
    assert r["n_clusters"] == 1 and r["n_clustered"] == n and np.all(r["label"] == 0)
    r = orc.cluster(xyz, t, d, [1], 0.4999, 2)
    assert r["n_clusters"] == 0 and np.all(r["label"] == 0xFFFFFFFF)
    r = orc.cluster(xyz, t, d, [1], 0.4999, 1)  # N_min = 1: every ion is its own cluster
    assert r["n_clusters"] == n and np.array_equal(r["label"], np.arange(n, dtype=np.uint32))
    # break the chain in the middle: two clusters of 20, labelled by their smallest index
    xyz[20:, 0] += np.float32(0.25)
    r = orc.cluster(xyz, t, d, [1], 0.5, 2)
    assert r["n_clusters"] == 2 and r["size_hist"][20] == 2
    assert np.all(r["label"][:20] == 0) and np.all(r["label"][20:] == 20)


def test_simple_cubic_lattice(orc, spec):
    xyz, t, d = spec.simple_cubic(10)  # a = 0.25 nm
    r = orc.cluster(xyz, t, d, [0], 0.25, 5)
    assert r["n_clusters"] == 1 and r["n_clustered"] == 1000 and r["size_hist"][1000] == 1
    r = orc.cluster(xyz, t, d, [0], 0.24, 1)
    assert r["n_clusters"] == 1000 and r["size_hist"][1] == 1000
    r = orc.cluster(xyz, t, d, [0], 0.24, 2)
    assert r["n_clusters"] == 0


def _brute(xyz, t, d, types, d_max, n_min, dsrf_min, hist_len):
    n = xyz.shape[0]
    D = np.float32(d_max * d_max)
    idx = np.nonzero(np.isin(t, types))[0]
    P = xyz[idx]
    rows, cols = [], []
    for a in range(idx.shape[0]):
        dd = P[a + 1:] - P[a]
        sq = dd * dd
        d2 = (sq[:, 0] + sq[:, 1]) + sq[:, 2]
        hit = np.nonzero(d2 <= D)[0] + a + 1
        rows += [a] * hit.shape[0]
        cols += hit.tolist()
    m = idx.shape[0]
    G = scipy_sparse.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(m, m))
    nc, comp = csgraph.connected_components(G, directed=False)
    size = np.bincount(comp, minlength=nc)
    cmin = np.full(nc, n, np.int64)
    np.minimum.at(cmin, comp, idx)
    dmin = np.full(nc, np.inf, np.float32)
    np.minimum.at(dmin, comp, d[idx])
    label = np.full(n, 0xFFFFFFFF, np.uint32)
    keep = size[comp] >= n_min
    label[idx[keep]] = cmin[comp[keep]]
    big = size >= n_min
    b = np.minimum(size[big], hist_len - 1)
    sh = np.bincount(b, minlength=hist_len)
    ih = np.bincount(b[dmin[big] >= dsrf_min], minlength=hist_len)
    return label, sh, ih, int(big.sum()), int(size[big].sum()), int((dmin[big] >= dsrf_min).sum())


@pytest.mark.parametrize("seed,d_max,n_min", [(1, 0.35, 3), (2, 0.5, 5), (3, 0.2, 1), (4, 0.6, 10)])
def test_brute_force_scipy(orc, seed, d_max, n_min):
    rng = np.random.default_rng(seed)
    n = 2500
    xyz = (rng.random((n, 3)) * 6.0).astype(np.float32)
    # a few dense blobs on top of the uniform background
    for c in rng.random((6, 3)) * 6.0:
        k = rng.integers(20, 80)
        xyz[rng.choice(n, k, replace=False)] = (c + rng.normal(0, 0.15, (k, 3))).astype(np.float32)
    t = rng.integers(0, 3, n).astype(np.uint8)
    d = (rng.random(n) * 2.0).astype(np.float32)
    hl = 64
    r = orc.cluster(xyz, t, d, [1, 2], d_max, n_min, 0.3, hl)
    label, sh, ih, ncl, nin, nint = _brute(xyz, t, d, [1, 2], d_max, n_min, np.float32(0.3), hl)
    np.testing.assert_array_equal(r["label"], label)
    np.testing.assert_array_equal(r["size_hist"].astype(np.int64), sh)
    np.testing.assert_array_equal(r["interior_hist"].astype(np.int64), ih)
    assert (r["n_clusters"], r["n_clustered"], r["n_interior"]) == (ncl, nin, nint)
    assert r["n_set"] == int(np.isin(t, [1, 2]).sum())


def test_partition_invariant_under_permutation(orc, spec):
    xyz, t, d = spec.cylinder(5, 4000, 3.0, 4.0, (0.5, 0.5))
    r = orc.cluster(xyz, t, d, [1], 0.45, 2)
    perm = np.random.default_rng(9).permutation(xyz.shape[0])
    rp = orc.cluster(xyz[perm], t[perm], d[perm], [1], 0.45, 2)
    np.testing.assert_array_equal(r["size_hist"], rp["size_hist"])
    la, lb = r["label"][perm], rp["label"]
    assert np.array_equal(la == 0xFFFFFFFF, lb == 0xFFFFFFFF)
    m = la != 0xFFFFFFFF
    # same partition: the map between the two labellings is a bijection
    pairs = set(zip(la[m].tolist(), lb[m].tolist()))
    assert len(pairs) == len(set(la[m].tolist())) == len(set(lb[m].tolist())) == r["n_clusters"]
