"""Pins for the spatial-distribution-map oracle (the 3-D two-point statistic):

* voxel edges that exact arithmetic fixes (V[n/2] = 0, V[n/2 + 10 i] = 0.25 i for w = 0.025);
* a simple-cubic lattice, where every interior central sees exactly one neighbour at each
  lattice vector shorter than R, on a voxel's lower edge (pins the half-open rule);
* an independent numpy brute force on small random clouds with displacements on edges;
* the map's total against the RDF pair count within R, and point symmetry of all-all maps.
"""
import numpy as np
import pytest


def _lattice(nc, a=0.25):
    g = (np.arange(nc, dtype=np.float64) * a + a / 2).astype(np.float32)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.float32)
    L = nc * a
    dsrf = np.minimum.reduce([xyz[:, 0], L - xyz[:, 0], xyz[:, 1], L - xyz[:, 1], xyz[:, 2], L - xyz[:, 2]])
    return xyz, np.ones(xyz.shape[0], np.uint8), dsrf.astype(np.float32)


def test_sdm_edges_exact(orc):
    V = orc.sdm_edges(0.025, 160)
    assert V.shape == (161,) and V.dtype == np.float32
    assert V[0] == np.float32(-2.0) and V[80] == np.float32(0.0) and V[160] == np.float32(2.0)
    for i in range(-8, 9):
        assert V[80 + 10 * i] == np.float32(0.25 * i)
    assert np.all(np.diff(V) > 0)


def test_sdm_simple_cubic_lattice(orc):
    xyz, t, d = _lattice(24)  # 6 nm block, a = 0.25 nm
    R, w, nv = 2.0, 0.025, 160
    H, meta = orc.sdm(xyz, t, d, [1], [1], R, R, w, nv)
    n_c = int((d >= np.float32(R)).sum())
    assert n_c > 0 and int(meta[0]) == n_c
    # lattice vectors (i, j, k) != 0 with (0.25)^2 (i^2 + j^2 + k^2) < R^2, by enumeration
    vecs = [(i, j, k) for i in range(-8, 9) for j in range(-8, 9) for k in range(-8, 9)
            if 0 < i * i + j * j + k * k < 64]
    want = np.zeros((nv, nv, nv), np.uint64)
    for i, j, k in vecs:
        want[80 + 10 * k, 80 + 10 * j, 80 + 10 * i] = n_c
    np.testing.assert_array_equal(H, want)
    assert int(meta[1]) == n_c * len(vecs) and int(meta[2]) == 0
    # the six unit vectors: displacement 0.25 lands on the lower edge of voxel 90, -0.25 on voxel 70
    assert H[80, 80, 90] == n_c and H[80, 80, 70] == n_c and H[80, 80, 89] == 0 and H[80, 80, 69] == 0


def _np_sdm(xyz, t, d, ctr, nbr, dmin, R, w, nv):
    """Independent numpy brute force: float32 displacements, searchsorted on the edges."""
    V = np.array([np.float32((m - nv / 2.0) * w) for m in range(nv + 1)], np.float32)
    ER = np.float32(R * R)
    H = np.zeros((nv, nv, nv), np.int64)
    inside = outside = n_c = 0
    nbr_idx = np.nonzero(np.isin(t, nbr))[0]
    for i in range(xyz.shape[0]):
        if t[i] not in ctr or not (d[i] >= dmin):
            continue
        n_c += 1
        j = nbr_idx[nbr_idx != i]
        dd = xyz[j] - xyz[i]
        sq = dd * dd
        d2 = (sq[:, 0] + sq[:, 1]) + sq[:, 2]
        dd = dd[d2 < ER]
        m = np.searchsorted(V, dd, side="right") - 1
        ok = np.all((dd >= V[0]) & (dd < V[-1]), axis=1)
        outside += int((~ok).sum())
        inside += int(ok.sum())
        np.add.at(H, (m[ok, 2], m[ok, 1], m[ok, 0]), 1)
    return H, (n_c, inside, outside)


@pytest.mark.parametrize("seed,nv,w", [(1, 40, 0.1), (2, 33, 0.125), (3, 16, 0.2)])
def test_sdm_numpy_brute_force(orc, seed, nv, w):
    rng = np.random.default_rng(seed)
    n = 700
    xyz = (rng.random((n, 3)) * 5.0).astype(np.float32)
    # a quarter of the points on a 0.025 nm grid: many displacements exactly on voxel edges
    q = rng.random(n) < 0.25
    xyz[q] = (np.round(xyz[q] / 0.025) * 0.025).astype(np.float32)
    t = rng.integers(0, 3, n).astype(np.uint8)
    d = (rng.random(n) * 3.0).astype(np.float32)
    R = 1.5
    H, meta = orc.sdm(xyz, t, d, [0, 1], [1, 2], 0.5, R, w, nv)
    Hn, mn = _np_sdm(xyz, t, d, [0, 1], [1, 2], 0.5, R, w, nv)
    np.testing.assert_array_equal(H.astype(np.int64), Hn)
    assert tuple(int(v) for v in meta) == mn
    if nv * w < 2 * R:
        assert mn[2] > 0  # the cube does not cover the ROI: some pairs fall outside
    else:
        assert mn[2] == 0


def test_sdm_total_equals_rdf_pairs_and_symmetry(orc):
    rng = np.random.default_rng(11)
    n = 3000
    # coordinates are odd multiples of 2^-13, so every displacement is a multiple of 2^-12
    xyz = ((np.floor(rng.random((n, 3)) * np.array([6.0, 5.0, 7.0]) * 4096) + 0.5) / 4096).astype(np.float32)
    t = rng.integers(0, 2, n).astype(np.uint8)
    d = np.full(n, 10.0, np.float32)
    R, w, nv = 1.2, 0.0500123, 49
    V = orc.sdm_edges(w, nv)
    # no edge is a multiple of 2^-12: no displacement lies on an edge
    assert not np.any(np.floor(V.astype(np.float64) * 4096) == V.astype(np.float64) * 4096)
    assert np.array_equal(V, -V[::-1])  # the edge table is symmetric about 0
    H, meta = orc.sdm(xyz, t, d, "all", "all", 0.0, R, w, nv)
    r = orc.spatstat(xyz, t, d, "all", "all", 0.0, 0.0, R, 1)
    assert int(meta[1]) + int(meta[2]) == r["n_pairs"] + r["rdf_below"]
    assert int(meta[2]) == 0 and int(H.sum()) == int(meta[1]) > 0
    # all-all with every ion central: each pair is seen from both ends, so the map is point symmetric
    np.testing.assert_array_equal(H, H[::-1, ::-1, ::-1])


def test_sdm_rejects_bad_arguments(orc):
    xyz = np.zeros((4, 3), np.float32)
    t = np.ones(4, np.uint8)
    d = np.zeros(4, np.float32)
    with pytest.raises(RuntimeError):
        orc.sdm(xyz, t, d, "all", "all", 0.0, 0.0, 0.1, 8)
    with pytest.raises(RuntimeError):
        orc.sdm(xyz, t, d, "all", "all", 0.0, 1.0, -0.1, 8)
