"""Pins of the oracle's g(r) normalisation (the RDF counts divided by the count a uniform
neighbour density puts in each shell about every central).  The paper gives no formula, so
the oracle follows a reading; these tests tie that reading to facts that do not depend on it:

* a homogeneous Poisson (binomial) process has g -> 1 at every radius: the mean over
  [0.5, 2] nm is 1 within 1 %, and every well-populated bin lies within its counting noise;
* g is invariant when the cloud, the specimen volume and the bins are scaled together by a
  power of two (exact in float32): a wrong exponent of the shell volume or of the density
  fails this;
* no centrals or no neighbours give g = 0 (not a division by zero)."""
import numpy as np


def _cube(spec, seed, rho, L, types=(1.0,)):
    n = int(round(rho * L**3))
    return spec.cube(seed, n, L, types), n


def test_poisson_g_tends_to_one(orc, spec):
    rho, L = 30.0, 13.0
    (xyz, t, d), n = _cube(spec, 41, rho, L)
    r0, dr, nb = 0.0, 0.05, 40
    r = orc.spatstat(xyz, t, d, "all", "all", 2.0, r0, dr, nb)
    g = orc.rdf_normalise(r["rdf"], r0, dr, r["n_central"], n, L**3)
    e = r0 + dr * np.arange(nb + 1)
    sel = e[:-1] >= 0.5
    assert abs(g[sel].mean() - 1.0) < 0.01
    # per bin: H_b is a count with variance ~2 E[H_b] (ordered pairs counted twice)
    expect = r["rdf"].astype(np.float64) / g.clip(1e-300)
    ok = expect >= 50
    assert ok.sum() > 30
    assert np.all(np.abs(g[ok] - 1.0) <= 6.0 * np.sqrt(2.0 / expect[ok]))


def test_poisson_g_with_disjoint_types(orc, spec):
    """Centrals of one type, neighbours of another: rho is the neighbour density alone."""
    rho, L = 40.0, 12.0
    (xyz, t, d), n = _cube(spec, 42, rho, L, (0.7, 0.3))
    r0, dr, nb = 0.0, 0.1, 20
    r = orc.spatstat(xyz, t, d, [1], [0], 2.0, r0, dr, nb)
    n_nbr = int((t == 0).sum())
    g = orc.rdf_normalise(r["rdf"], r0, dr, r["n_central"], n_nbr, L**3)
    e = r0 + dr * np.arange(nb + 1)
    assert abs(g[e[:-1] >= 0.5].mean() - 1.0) < 0.015


def test_g_invariant_under_joint_scaling(orc, spec):
    (xyz, t, d), n = _cube(spec, 43, 30.0, 9.0)
    base = orc.spatstat(xyz, t, d, "all", "all", 1.5, 0.0, 0.02, 75)
    g0 = orc.rdf_normalise(base["rdf"], 0.0, 0.02, base["n_central"], n, 9.0**3)
    for c in (0.5, 2.0, 4.0):
        xs, ds = (xyz * np.float32(c)).astype(np.float32), (d * np.float32(c)).astype(np.float32)
        r = orc.spatstat(xs, t, ds, "all", "all", 1.5 * c, 0.0, 0.02 * c, 75)
        np.testing.assert_array_equal(r["rdf"], base["rdf"])  # power-of-two scaling is exact
        g = orc.rdf_normalise(r["rdf"], 0.0, 0.02 * c, r["n_central"], n, (9.0 * c) ** 3)
        np.testing.assert_allclose(g, g0, rtol=1e-12, atol=0)


def test_empty_sets_give_zero(orc):
    h = np.arange(10, dtype=np.uint64)
    assert np.all(orc.rdf_normalise(h, 0.0, 0.1, 0, 100, 10.0) == 0.0)
    assert np.all(orc.rdf_normalise(h, 0.0, 0.1, 100, 0, 10.0) == 0.0)
