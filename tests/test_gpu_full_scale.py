"""Full-size parity on the 2e9-ion needle (tip radius 40 nm, half-angle 15 deg, 30 ions/nm^3).

* all-all, k = 10, RDF on r = [0, 0.01, 2] nm, d_srf >= 2 nm, on the whole cloud with
  per-central outputs: properties that hold at any size (counts consistent between the
  histograms and the per-central outputs, the kNN histogram equal to the binned per-central
  k-th distances, the central count equal to the d_srf rule applied on the host) and 32
  sampled centrals against the oracle's brute force over the whole cloud;
* all-all, every bin: three z-slabs of centrals -- at the tip, at mid-height and at the base,
  ~0.2-2.5e6 centrals each -- selected on the GPU by a d_srf array that disqualifies every
  other ion (NaN), queried on the grid of the whole 2e9-ion cloud, against the oracle run on
  that slab plus an r_cut halo of neighbours (split into x-strips over the host cores, which
  add up exactly): the RDF, kNN, not-found and pair counts bin for bin, and the full-size
  run's per-central k-th distance and in-range count of every slab central;
* Sc-Sc, k = 10, same bins and d_srf: the complete oracle, every bin;
* the launch configuration the benchmark times (half-size cells, the query in passes): the
  whole-cloud all-all histograms equal to the 27-cell run's bin for bin, the three slabs against
  the same oracle results, and Sc-Sc against the complete oracle, with and without the passes.

Needs ~40 GB of host memory and ~190 GB of device memory; takes a few minutes.
"""
import concurrent.futures as cf
import os
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if free < 190 * 2**30:
        pytest.skip("needs ~190 GB of free device memory")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2004_05188_gb300 as ps

    return ps


def _oracle_slab(orc, xyz, t, d, lo, hi, r_cut, bins, ks, threads):
    """The oracle on the centrals with index in [lo, hi): x-strips of equal central count, each
    with every ion of [lo, hi)'s neighbourhood within r_cut of the strip in x; summed.
    Returns the summed result and the per-central outputs of the centrals (index, kth, n_within)."""
    x = xyz[:, 0]
    cx = np.sort(x[lo:hi])
    cuts = [-np.inf] + [float(cx[len(cx) * j // threads]) for j in range(1, threads)] + [np.inf]

    def one(j):
        keep = np.nonzero((x >= cuts[j] - r_cut) & (x < cuts[j + 1] + r_cut))[0]
        own = (keep >= lo) & (keep < hi) & (x[keep] >= cuts[j]) & (x[keep] < cuts[j + 1])
        dj = np.where(own, d[keep], np.float32(np.nan)).astype(np.float32)
        r = orc.spatstat(xyz[keep], t[keep], dj, "all", "all", 2.0, *bins, ks, per_central=True)
        c = np.nonzero(own & (dj >= np.float32(2.0)))[0]
        return r, keep[c], r["kth_d2"][0][c], r["n_within"][c]

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, range(threads)))
    tot = {k: sum(r[0][k] for r in res) for k in ("rdf", "knn")}
    tot["n_central"] = sum(r[0]["n_central"] for r in res)
    tot["n_pairs"] = sum(r[0]["n_pairs"] for r in res)
    tot["not_found"] = sum(np.asarray(r[0]["not_found"]) for r in res)
    idx = np.concatenate([r[1] for r in res])
    return tot, idx, np.concatenate([r[2] for r in res]), np.concatenate([r[3] for r in res])


def test_needle_2e9_full_size(ps, orc, spec):
    t0 = time.perf_counter()
    p = spec.needle_2g_params()
    counts = spec.needle_plan(p)
    n = int(counts.sum())
    xyz = np.empty((n, 3), np.float32)
    t = np.empty(n, np.uint8)
    d = np.empty(n, np.float32)
    spec.needle_fill(p, 0, counts.shape[0], counts, xyz.ctypes.data, t.ctypes.data, d.ctypes.data)
    gen_s = time.perf_counter() - t0
    assert 1.95e9 < n < 2.05e9
    X = torch.from_numpy(xyz).cuda()
    T = torch.from_numpy(t).cuda()
    D = torch.from_numpy(d).cuda()
    bins = ps.bins_from_spec(0.0, 0.01, 2.0)
    E = ps.edges(*bins)

    g = ps.Grid(n)
    # ---- all-all, k = 10, whole cloud ----
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    g.build(X, T, "all", 2.0)
    out = ps.spatstat(g, D, "all", 2.0, bins, [10], per_central=True)
    torch.cuda.synchronize()
    gpu_s = time.perf_counter() - t1
    meta = out["meta"].cpu().numpy()
    assert meta[3] == 0
    n_c = int(meta[0])
    central = d >= np.float32(2.0)
    assert n_c == int(central.sum())
    rdf = out["rdf"].cpu().numpy()
    knn_all = out["knn"].cpu().numpy()
    knn = knn_all[0]
    nw = out["n_within"]
    kth = out["kth_d2"][0]
    Cm = torch.from_numpy(central).cuda()
    assert int(rdf.sum()) == int(meta[1]) == int(nw[Cm].sum(dtype=torch.int64).item())
    assert int(knn.sum()) + int(meta[4]) + int(meta[5]) == n_c
    assert bool((nw[~Cm] == -1).all().item()) and bool(torch.isnan(kth[~Cm]).all().item())
    kc = kth[Cm]
    found = kc[torch.isfinite(kc)]
    assert found.numel() == n_c - int(meta[4])
    Et = torch.from_numpy(E).cuda()
    b = torch.bucketize(found, Et, right=True, out_int32=True) - 1
    np.testing.assert_array_equal(torch.bincount(b, minlength=bins[2]).cpu().numpy()[: bins[2]], knn)
    kth_h = kth.cpu().numpy()
    nw_h = nw.cpu().numpy()
    del out, kth, nw, kc, found, b, Cm
    threads = os.cpu_count() or 8

    # sampled centrals against the oracle's brute force over all n ions (threads: ctypes releases the GIL)
    rng = np.random.default_rng(2024)
    samples = rng.choice(np.nonzero(central)[0], 32, replace=False)

    def one(i):
        return orc.central_brute(xyz, t, int(i), "all", *bins, [10])

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(one, samples))
    for i, (nwi, kthi, _) in zip(samples, res):
        assert nw_h[i] == nwi
        assert kth_h[i] == kthi[0] or (np.isinf(kth_h[i]) and np.isinf(kthi[0]))

    # ---- all-all, every bin: slabs of centrals at the tip, mid-height and the base ----
    off = np.concatenate([[0], np.cumsum(counts)])
    nk = counts.shape[0]
    # layers ~0.4 nm high; the base slab starts above z = 4 nm (the bottom face's d_srf < 2 nm below)
    slabs = {"tip": (nk - 40, nk - 8), "mid": (nk // 2, nk // 2 + 2), "base": (10, 11)}
    halo = 16  # layers: 6.5 nm > r_cut + the z jitter on both sides
    Dm = torch.empty_like(D)
    refs = {}
    for name, (k0, k1) in slabs.items():
        lo, hi = int(off[k0]), int(off[k1])
        a, z = int(off[max(0, k0 - halo)]), xyz[:, 2]
        e = int(off[min(nk, k1 + halo)])
        zc = z[lo:hi]
        # the halo holds every neighbour within r_cut of the slab's ions (checked on the whole cloud)
        for part in (z[:a], z[e:]):
            assert not np.any((part > zc.min() - 2.0) & (part < zc.max() + 2.0)), name
        Dm.fill_(float("nan"))
        Dm[lo:hi] = D[lo:hi]
        o = ps.spatstat(g, Dm, "all", 2.0, bins, [10])
        ref, idx, kref, nref = _oracle_slab(orc, xyz[a:e], t[a:e], d[a:e], lo - a, hi - a, 2.0, bins, [10], threads)
        refs[name] = (lo, hi, ref)
        m = o["meta"].cpu().numpy()
        assert m[3] == 0 and ref["n_central"] > 1e5, (name, ref["n_central"])
        assert m[0] == ref["n_central"] and m[1] == ref["n_pairs"] and m[4] == ref["not_found"][0], name
        np.testing.assert_array_equal(o["rdf"].cpu().numpy().astype(np.uint64), ref["rdf"])
        np.testing.assert_array_equal(o["knn"].cpu().numpy().astype(np.uint64), ref["knn"])
        # the full-size run's per-central outputs of these centrals
        np.testing.assert_array_equal(nw_h[idx + a], nref)
        np.testing.assert_array_equal(kth_h[idx + a], kref)
        print(f"\n  {name} slab: {ref['n_central']} centrals, {ref['n_pairs']} pairs, every bin equal")

    # ---- Sc-Sc, k = 10: the complete oracle ----
    g.build(X, T, [1], 2.0)
    o = ps.spatstat(g, D, [1], 2.0, bins, [10])
    r = orc.spatstat(xyz, t, d, [1], [1], 2.0, *bins, [10])

    def same_as_oracle(o, r, what):
        np.testing.assert_array_equal(o["rdf"].cpu().numpy().astype(np.uint64), r["rdf"], err_msg=what)
        np.testing.assert_array_equal(o["knn"].cpu().numpy().astype(np.uint64), r["knn"], err_msg=what)
        m = o["meta"].cpu().numpy()
        assert m[3] == 0 and m[0] == r["n_central"] and m[1] == r["n_pairs"] and m[4] == r["not_found"][0], what

    same_as_oracle(o, r, "Sc-Sc")
    g.close()

    # ---- the benchmark's launch configuration: half-size cells, the query in passes ----
    g = ps.Grid(n, 0.5, 0, True)
    g.build(X, T, "all", 2.0)
    o = ps.spatstat(g, D, "all", 2.0, bins, [10])
    np.testing.assert_array_equal(o["rdf"].cpu().numpy(), rdf)
    np.testing.assert_array_equal(o["knn"].cpu().numpy(), knn_all)
    np.testing.assert_array_equal(o["meta"].cpu().numpy(), meta)
    for name, (lo, hi, ref) in refs.items():
        Dm.fill_(float("nan"))
        Dm[lo:hi] = D[lo:hi]
        same_as_oracle(ps.spatstat(g, Dm, "all", 2.0, bins, [10]), ref, name + " slab, passes")
    del Dm
    g.build(X, T, [1], 2.0)
    for split in (False, True):
        g.set_query_opts(0, split)
        same_as_oracle(ps.spatstat(g, D, [1], 2.0, bins, [10]), r, f"Sc-Sc, half-size cells, split={split}")
    g.close()
    print(f"\n2e9 needle: n={n}, generation {gen_s:.1f} s, all-all build+query {gpu_s:.1f} s, "
          f"{n_c} centrals, {int(meta[1])} pairs, Sc-Sc centrals {r['n_central']}")
