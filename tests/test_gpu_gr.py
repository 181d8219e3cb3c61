"""GPU parity of the g(r) finalisation (ps_rdf_normalise) against the oracle's FP64 formula.

The counts come from the exact path (bit-identical to the oracle's, checked here again), |C|
from the query's meta array and |N| from the grid on the device; g and the per-bin factor
must equal the oracle's FP64 values to within a few units of the last place (both sides
evaluate the same expression in IEEE double, round to nearest)."""
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


CASES = [
    # cloud, central types, neighbour types, d_srf threshold, bins, volume
    ("cylinder", "all", "all", 1.0, (0.0, 0.01, 200)),
    ("cylinder", [1], [0], 2.0, (0.0, 0.02, 100)),
    ("cylinder", [0, 2], [1, 2], 0.5, (0.3, 0.05, 34)),
    ("cube", "all", "all", 2.0, (0.0, 0.05, 40)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_rdf_normalise_matches_oracle(ps, orc, spec, case):
    cloud, ctr, nbr, dmin, bins = CASES[case]
    if cloud == "cylinder":
        xyz, t, d = spec.cylinder(51, 150_000, 10.0, 12.0)
        vol = math.pi * 10.0**2 * 12.0
    else:
        xyz, t, d = spec.cube(52, 60_000, 13.0, (1.0,))
        vol = 13.0**3
    X, T, D = (torch.from_numpy(a).cuda() for a in (xyz, t, d))
    r0, dr, nb = bins
    g = ps.Grid(X.shape[0]).build(X, T, nbr, float(np.float32(r0 + nb * dr)) * (1 + 1e-6))
    out = ps.spatstat(g, D, ctr, dmin, bins, [])
    gg, f = ps.rdf_normalise(g, out["meta"], bins, vol, rdf=out["rdf"])
    _, f_only = ps.rdf_normalise(g, out["meta"], bins, vol)
    torch.cuda.synchronize()
    ref = orc.spatstat(xyz, t, d, ctr, nbr, dmin, r0, dr, nb)
    np.testing.assert_array_equal(out["rdf"].cpu().numpy().astype(np.uint64), ref["rdf"])
    n_nbr = int(np.isin(t, np.arange(256) if nbr == "all" else nbr).sum())
    g_ref = orc.rdf_normalise(ref["rdf"], r0, dr, ref["n_central"], n_nbr, vol)
    np.testing.assert_allclose(gg.cpu().numpy(), g_ref, rtol=4e-16 * 8, atol=0)
    np.testing.assert_array_equal(f.cpu().numpy(), f_only.cpu().numpy())
    np.testing.assert_allclose(f.cpu().numpy() * ref["rdf"].astype(np.float64), g_ref, rtol=1e-14, atol=0)
    if cloud == "cube":
        e = r0 + dr * np.arange(nb + 1)
        assert abs(gg.cpu().numpy()[e[:-1] >= 0.5].mean() - 1.0) < 0.01  # Poisson: g -> 1
    g.close()
