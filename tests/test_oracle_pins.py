"""Pins for the exact kNN / RDF oracle: checks against things other than itself.

* edge table values fixed by exact arithmetic and the paper's bin notation;
* O(N^2) brute force (C) and an independent numpy brute force on small clouds;
* exact neighbour shells of a simple-cubic lattice (r3(n) by enumeration);
* closed-form expectations of the homogeneous binomial point process.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _np_brute(xyz, type_, dsrf, ctr, nbr, dsrf_min, E, ks):
    """Independent numpy brute force: float32 ops in the fixed order, searchsorted on E."""
    xyz = xyz.astype(np.float32)
    n = xyz.shape[0]
    nb = E.shape[0] - 1
    rdf = np.zeros(nb, np.int64)
    knn = np.zeros((len(ks), nb), np.int64)
    nf = np.zeros(len(ks), np.int64)
    n_central = 0
    nbr_idx = np.nonzero(np.isin(type_, list(nbr)))[0]
    for i in range(n):
        if type_[i] not in ctr or not (dsrf[i] >= dsrf_min):
            continue
        n_central += 1
        j = nbr_idx[nbr_idx != i]
        d = xyz[j] - xyz[i]  # float32 subtraction
        sq = d * d  # float32 products
        d2 = (sq[:, 0] + sq[:, 1]) + sq[:, 2]  # float32 sums, fixed order
        d2 = d2[d2 < E[-1]]
        b = np.searchsorted(E, d2, side="right") - 1
        rdf += np.bincount(b[b >= 0], minlength=nb)
        s = np.sort(d2)
        for q, k in enumerate(ks):
            if s.shape[0] < k:
                nf[q] += 1
            else:
                bk = np.searchsorted(E, s[k - 1], side="right") - 1
                if bk >= 0:
                    knn[q, bk] += 1
    return rdf, knn, nf, n_central


def test_edge_table_exact_values(orc):
    E = orc.edges(0.0, 0.01, 200)
    assert E.dtype == np.float32 and E.shape == (201,)
    # e_b = b * 0.01 squared: these edges are exactly representable
    assert E[0] == np.float32(0.0)
    assert E[25] == np.float32(0.0625)
    assert E[50] == np.float32(0.25)
    assert E[75] == np.float32(0.5625)
    assert E[100] == np.float32(1.0)
    assert E[200] == np.float32(4.0)
    assert np.all(np.diff(E) > 0)
    # a float32 step gives a different table at 111 of the 201 edges (e.g. b = 5, 10, 20):
    # r0 and dr are double in the contract
    Ef = (np.float32(0.01) * np.arange(201, dtype=np.float32)) ** 2
    assert int((Ef != E).sum()) == 111 and Ef[10] != E[10]
    # non-zero start
    E2 = orc.edges(0.5, 0.25, 6)
    assert list(E2) == [0.25, 0.5625, 1.0, 1.5625, 2.25, 3.0625, 4.0]


def test_paper_bin_specs(orc):
    from paper_2004_05188_gb300 import bins_from_spec

    with open(os.path.join(GOLDEN, "paper_bin_specs.txt")) as f:
        rows = [ln.split()[:4] for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 2
    for start, step, stop, n in rows:
        r0, dr, nb = bins_from_spec(float(start), float(step), float(stop))
        assert nb == int(n)
        E = orc.edges(r0, dr, nb)
        assert E[-1] == np.float32(float(stop) ** 2)


@pytest.mark.parametrize("n,L,seed", [(1000, 6.0, 11), (4000, 9.0, 12)])
def test_cell_list_equals_brute_force(orc, spec, n, L, seed):
    xyz, t, d = spec.cube(seed, n, L, (0.6, 0.3, 0.1))
    for ctr, nbr, dmin, ks in [("all", "all", 0.0, [1, 2, 7]), ([1], [1], 1.0, [1, 3]), ([0], [1, 2], 0.5, [1]),
                               ([2], "all", -1.0, [4, 32])]:
        a = orc.spatstat(xyz, t, d, ctr, nbr, dmin, 0.0, 0.02, 100, ks, per_central=True)
        b = orc.spatstat(xyz, t, d, ctr, nbr, dmin, 0.0, 0.02, 100, ks, per_central=True, brute=True)
        for key in ("rdf", "knn", "not_found", "knn_below"):
            np.testing.assert_array_equal(a[key], b[key])
        assert a["n_central"] == b["n_central"] and a["n_pairs"] == b["n_pairs"]
        np.testing.assert_array_equal(a["kth_d2"], b["kth_d2"])
        np.testing.assert_array_equal(a["n_within"], b["n_within"])


def test_oracle_equals_numpy_brute_force(orc, spec):
    xyz, t, d = spec.cube(21, 1500, 7.0, (0.5, 0.5))
    E = orc.edges(0.0, 0.01, 150)
    for ctr, nbr, dmin, ks in [({0, 1}, {0, 1}, 1.0, [1, 5]), ({1}, {0}, 0.0, [2])]:
        rdf, knn, nf, nc = _np_brute(xyz, t, d, ctr, nbr, dmin, E, ks)
        a = orc.spatstat(xyz, t, d, sorted(ctr), sorted(nbr), dmin, 0.0, 0.01, 150, ks)
        np.testing.assert_array_equal(a["rdf"].astype(np.int64), rdf)
        np.testing.assert_array_equal(a["knn"].astype(np.int64), knn)
        np.testing.assert_array_equal(a["not_found"].astype(np.int64), nf)
        assert a["n_central"] == nc


def test_cylinder_subsample_brute(orc, spec):
    xyz, t, d = spec.cylinder_small()
    sel = np.random.default_rng(3).choice(xyz.shape[0], 6000, replace=False)
    sel.sort()
    x, ty, ds = xyz[sel], t[sel], d[sel]
    a = orc.spatstat(x, ty, ds, "all", "all", 1.0, 0.0, 0.01, 200, [1, 3], per_central=True)
    b = orc.spatstat(x, ty, ds, "all", "all", 1.0, 0.0, 0.01, 200, [1, 3], per_central=True, brute=True)
    for key in ("rdf", "knn", "not_found", "kth_d2", "n_within"):
        np.testing.assert_array_equal(a[key], b[key])


def test_duplicates_and_points_on_edges(orc):
    # coincident distinct ions count at d = 0 (bin 0) and as neighbours; the self pair never counts
    xyz = np.array([[1, 1, 1], [1, 1, 1], [1.25, 1, 1], [1, 1.5, 1], [3, 3, 3]], np.float32)
    t = np.zeros(5, np.uint8)
    d = np.full(5, 10.0, np.float32)
    r = orc.spatstat(xyz, t, d, "all", "all", 0.0, 0.0, 0.01, 100, [1, 2, 3], per_central=True)
    # pairs (ordered): 0-1 and 1-0 at d=0; 0-2, 1-2 at 0.25 (edge 25); 0-3, 1-3 at 0.5 (edge 50);
    # 2-3 at sqrt(0.0625+0.25)=0.559..; ion 4 has nobody within 1 nm
    assert r["rdf"][0] == 2
    assert r["rdf"][25] == 4 and r["rdf"][24] == 0
    assert r["rdf"][50] == 4 and r["rdf"][49] == 0
    assert r["rdf"][55] == 2
    assert r["n_central"] == 5 and r["n_pairs"] == 12
    assert list(r["n_within"]) == [3, 3, 3, 3, 0]
    assert r["kth_d2"][0, 0] == 0.0 and r["kth_d2"][0, 1] == 0.0
    assert r["kth_d2"][0, 2] == np.float32(0.0625)
    assert r["not_found"][0] == 1 and r["not_found"][2] == 1
    assert np.isinf(r["kth_d2"][0, 4])


def _r3(nmax):
    """number of integer triples with i^2+j^2+k^2 = n, by enumeration"""
    c = np.zeros(nmax + 1, np.int64)
    m = int(math.isqrt(nmax)) + 1
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            for k in range(-m, m + 1):
                s = i * i + j * j + k * k
                if s <= nmax:
                    c[s] += 1
    return c


def test_simple_cubic_shells(orc, spec):
    # a = 0.25 nm: every squared distance n/16 is exact in float32
    xyz, t, d = spec.simple_cubic(24, 0.25, 0.125)
    r = orc.spatstat(xyz, t, d, "all", "all", 2.0, 0.0, 0.01, 200, list(range(1, 33)), per_central=True)
    nc = r["n_central"]
    assert nc == 8**3  # coordinates 0.125 + 0.25 i in [2, 4]
    r3 = _r3(63)
    expect = np.zeros(200, np.int64)
    for n in range(1, 64):  # d < 2 nm  <=>  n < 64
        b = math.isqrt(625 * n)  # largest b with (b/100)^2 <= n/16
        expect[b] += nc * r3[n]
    np.testing.assert_array_equal(r["rdf"].astype(np.int64), expect)
    # the lower-inclusive rule on exact edges: n = 1, 4, 9, 16 land on edges 25, 50, 75, 100
    assert r["rdf"][25] == nc * 6 and r["rdf"][24] == 0
    assert r["rdf"][50] == nc * 6 and r["rdf"][100] == nc * 6
    # kNN: shells 6, 12, 8, 6 at n = 1, 2, 3, 4
    shell_of_k = np.repeat([1, 2, 3, 4], [6, 12, 8, 6])
    cent = r["kth_d2"][:, ~np.isnan(r["kth_d2"][0])]
    for k in range(1, 33):
        assert np.all(cent[k - 1] == np.float32(shell_of_k[k - 1] / 16.0))
        b = math.isqrt(625 * int(shell_of_k[k - 1]))
        assert r["knn"][k - 1, b] == nc and r["knn"][k - 1].sum() == nc
    assert np.all(r["not_found"] == 0)


def _poisson_cloud(spec, seed, rho, L):
    n = int(round(rho * L**3))
    return spec.cube(seed, n, L, (1.0,)), n


def test_poisson_rdf_closed_form(orc, spec):
    """Binomial process in a cube: E[H_b] = |C| (N-1)/V * 4/3 pi (e_{b+1}^3 - e_b^3)."""
    rho, L, rmax = 30.0, 13.0, 2.0
    (xyz, t, d), n = _poisson_cloud(spec, 31, rho, L)
    r = orc.spatstat(xyz, t, d, "all", "all", rmax, 0.0, 0.05, 40)
    nc = r["n_central"]
    e = np.arange(41) * 0.05
    Eh = nc * (n - 1) / L**3 * 4.0 / 3.0 * np.pi * (e[1:] ** 3 - e[:-1] ** 3)
    H = r["rdf"].astype(np.float64)
    ok = Eh >= 50
    assert ok.sum() > 30
    assert np.all(np.abs(H[ok] - Eh[ok]) <= 6.0 * np.sqrt(2.0 * Eh[ok]))
    g = H / Eh
    sel = e[:-1] >= 0.5
    assert abs(g[sel].mean() - 1.0) < 0.01


def test_poisson_knn_closed_form(orc, spec):
    """k-th NN distance of an interior point: P(R_k <= r) = P(Binomial(N-1, 4/3 pi r^3 / V) >= k)."""
    from scipy.stats import binom

    rho, L, rmax = 30.0, 13.0, 2.0
    (xyz, t, d), n = _poisson_cloud(spec, 32, rho, L)
    ks = [1, 5, 10]
    r = orc.spatstat(xyz, t, d, "all", "all", rmax, 0.0, 0.01, 200, ks)
    nc = r["n_central"]
    e = np.arange(201) * 0.01
    p = 4.0 / 3.0 * np.pi * e**3 / L**3
    for q, k in enumerate(ks):
        cdf = binom.sf(k - 1, n - 1, p)
        expect = nc * np.diff(cdf)
        obs = r["knn"][q].astype(np.float64)
        ok = expect >= 5
        df = int(ok.sum()) - 1
        chi2 = float(np.sum((obs[ok] - expect[ok]) ** 2 / expect[ok]))
        assert chi2 / df <= 1.0 + 6.0 * math.sqrt(2.0 / df), (k, chi2 / df)
        assert r["not_found"][q] == 0
    # the density of the paper's closed form integrates to the same CDF (Poisson limit)
    lam = 4.0 / 3.0 * np.pi * rho * e**3
    for k in ks:
        pois = 1.0 - sum(np.exp(-lam) * lam**j / math.factorial(j) for j in range(k))
        assert np.max(np.abs(pois - binom.sf(k - 1, n - 1, p))) < 2e-3
