"""Randomised labels on the GPU: identical to the oracle's permutation, and the statistics on them."""
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


@pytest.mark.parametrize("n,seed", [(1, 3), (5, 3), (100_003, 11), (2_000_000, 2**63 + 5)])
def test_permutation_equals_oracle(ps, orc, n, seed):
    t = np.random.default_rng(n).integers(0, 256, n).astype(np.uint8)
    out, perm = ps.shuffle_labels(torch.from_numpy(t).cuda(), seed, with_perm=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(perm.cpu().numpy().astype(np.uint32), orc.label_perm(n, seed))
    np.testing.assert_array_equal(out.cpu().numpy(), orc.shuffle_labels(t, seed))


def test_statistics_on_randomised_labels(ps, orc, spec):
    """Sc-Sc on the 1e6-ion needle ROI with shuffled labels: equal to the oracle on the same labels,
    and the clustering of the precipitates is gone (the RDF follows the all-all RDF scaled by the
    Sc pair fraction)."""
    xyz, t, d = spec.roi(0, 1_000_000)
    X, T, D = (torch.from_numpy(a).cuda() for a in (xyz, t, d))
    Tr = ps.shuffle_labels(T, 2020)
    tr = orc.shuffle_labels(t, 2020)
    np.testing.assert_array_equal(Tr.cpu().numpy(), tr)
    bins = (0.0, 0.05, 40)
    g = ps.Grid(X.shape[0]).build(X, Tr, [1], 2.0)
    o = ps.spatstat(g, D, [1], 2.0, bins, [1, 5])
    r = orc.spatstat(xyz, tr, d, [1], [1], 2.0, *bins, [1, 5])
    np.testing.assert_array_equal(o["rdf"].cpu().numpy().astype(np.uint64), r["rdf"])
    np.testing.assert_array_equal(o["knn"].cpu().numpy().astype(np.uint64), r["knn"])
    ga = ps.Grid(X.shape[0]).build(X, Tr, "all", 2.0)
    oa = ps.spatstat(ga, D, "all", 2.0, bins, [])
    n, n_sc = t.shape[0], int((t == 1).sum())
    frac = n_sc / n * (n_sc - 1) / (n - 1)
    H = o["rdf"].cpu().numpy().astype(np.float64)
    Ha = oa["rdf"].cpu().numpy().astype(np.float64) * frac
    ok = Ha >= 100
    assert ok.sum() > 20
    assert np.all(np.abs(H[ok] - Ha[ok]) <= 6 * np.sqrt(2 * Ha[ok]))
    # the original labels are clustered: many more short Sc-Sc pairs than random
    go = ps.Grid(X.shape[0]).build(X, T, [1], 2.0)
    oo = ps.spatstat(go, D, [1], 2.0, bins, [])
    assert oo["rdf"][:10].sum().item() > 3 * o["rdf"][:10].sum().item()
    for gg in (g, ga, go):
        gg.close()
