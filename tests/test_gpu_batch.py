"""The batched sweep against the plain per-ROI exact path, bit for bit (and one ROI against the oracle)."""
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


def _rois(spec):
    rois = [spec.cylinder(71, 3000, 4.0, 6.0), spec.cube(72, 20000, 9.0, (0.7, 0.25, 0.05)),
            spec.roi(0, 12000), spec.roi(1, 8000), spec.cube(73, 40, 3.0, (0.5, 0.5)), spec.roi(2, 30000)]
    return [tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in r) for r in rois], rois


@pytest.mark.parametrize("cell_scale", [1.0, 0.5])
def test_batched_equals_plain_calls(ps, spec, cell_scale):
    dev_rois, _ = _rois(spec)
    bins = (0.0, 0.01, 150)
    rmax_bins = [50, 100, 150]
    dsrf_min = [0.0, 0.5, 1.0]
    pairs = [("all", "all"), ([1], [1]), ([0], [1])]
    k_max = 20
    b = ps.Batch(dev_rois, bins, rmax_bins, dsrf_min, pairs, k_max, cell_scale)
    out = b.run()
    out2 = b.run()  # a second run must give the same result (accumulators are cleared)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
    rdf, knn, meta = b.split(out.cpu().numpy())
    ks = list(range(1, k_max + 1))
    for i, (X, T, D) in enumerate(dev_rois):
        for p, (ctr, nbr) in enumerate(pairs):
            for r, nbr_ in enumerate(rmax_bins):
                g = ps.Grid(X.shape[0]).build(X, T, nbr, nbr_ * 0.01 * (1 + 1e-6))
                for q, dmin in enumerate(dsrf_min):
                    o = ps.spatstat(g, D, ctr, dmin, (0.0, 0.01, nbr_), ks)
                    np.testing.assert_array_equal(rdf[i, p, r, q, :nbr_], o["rdf"].cpu().numpy())
                    assert np.all(rdf[i, p, r, q, nbr_:] == 0)
                    np.testing.assert_array_equal(knn[i, p, r, q, :, :nbr_], o["knn"].cpu().numpy())
                    np.testing.assert_array_equal(meta[i, p, r, q], o["meta"].cpu().numpy())
                g.close()
    b.close()


def test_batched_one_roi_against_oracle(ps, orc, spec):
    dev_rois, host = _rois(spec)
    b = ps.Batch(dev_rois[1:2], (0.0, 0.02, 75), [75], [0.0, 1.0], [("all", "all"), ([1], [0, 2])], 5)
    rdf, knn, meta = b.split(b.run().cpu().numpy())
    xyz, t, d = host[1]
    for p, (ctr, nbr) in enumerate([("all", "all"), ([1], [0, 2])]):
        for q, dmin in enumerate([0.0, 1.0]):
            r = orc.spatstat(xyz, t, d, ctr, nbr, dmin, 0.0, 0.02, 75, [1, 2, 3, 4, 5])
            np.testing.assert_array_equal(rdf[0, p, 0, q].astype(np.uint64), r["rdf"])
            np.testing.assert_array_equal(knn[0, p, 0, q].astype(np.uint64), r["knn"])
            assert meta[0, p, 0, q, 0] == r["n_central"]
            np.testing.assert_array_equal(meta[0, p, 0, q, 4::2].astype(np.uint64), r["not_found"])
    b.close()


def test_batched_256_rois_full_size_sampled(ps, spec):
    """The full batched workload (256 ROIs, log-uniform 1e4..1e7 ions, k = 1..20, r_max {1,2,3} nm,
    d_srf {0,1,2} nm, all-all / Sc-Sc / Al-Sc) in one run; 12 sampled (ROI, pair, r_max, d_srf)
    records against the plain exact call, bit for bit."""
    sizes = spec.roi_sizes(256)
    rois = [tuple(torch.from_numpy(a).cuda() for a in spec.roi(i, n)) for i, n in enumerate(sizes)]
    bins, rmax, dsrf = (0.0, 0.01, 300), [100, 200, 300], [0.0, 1.0, 2.0]
    pairs, k_max = [("all", "all"), ([1], [1]), ([0], [1])], 20
    b = ps.Batch(rois, bins, rmax, dsrf, pairs, k_max, 0.5)
    out = b.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    picks = [(int(rng.integers(256)), int(rng.integers(3)), int(rng.integers(3)), int(rng.integers(3)))
             for _ in range(12)]
    picks.append((int(np.argmax(sizes)), 0, 2, 0))  # the largest ROI, all-all, r_max 3, d_srf >= 0
    ks = list(range(1, k_max + 1))
    for i, p, r, q in picks:
        X, T, D = rois[i]
        ctr, nbr = pairs[p]
        g = ps.Grid(X.shape[0]).build(X, T, nbr, rmax[r] * 0.01 * (1 + 1e-6))
        o = ps.spatstat(g, D, ctr, dsrf[q], (0.0, 0.01, rmax[r]), ks)
        rdf, knn, meta = b.split(out[i, p, r, q].cpu().numpy())
        np.testing.assert_array_equal(rdf[: rmax[r]], o["rdf"].cpu().numpy())
        np.testing.assert_array_equal(knn[:, : rmax[r]], o["knn"].cpu().numpy())
        np.testing.assert_array_equal(meta, o["meta"].cpu().numpy())
        g.close()
    b.close()
