"""Pins for the FP64 Gaussian-smoothed RDF oracle and its adjoint.

* sigma -> 0: the smoothed histogram becomes the exact integer histogram;
* telescoping: sum_b h[b] = sum over pairs of Phi((stop-u)/sigma) - Phi((r0-u)/sigma);
* the adjoint against central finite differences of the forward;
* translation invariance (sum_i dL/dx_i = 0) and the Euler scaling identity
  s dL/ds = sum_i x_i . dL/dx_i (every pair distance scales with s).
"""
import numpy as np
from scipy.special import ndtr

SIG, R0, DR, NB = 0.05, 0.0, 0.02, 100


def _cloud(spec, seed, n, L, probs=(0.7, 0.3)):
    return spec.cube(seed, n, L, probs)


def _pairs(xyz, t, d, ctr, nbr, dmin):
    x = xyz.astype(np.float64)
    cen = np.nonzero(np.isin(t, ctr) & (d >= dmin))[0]
    nb = np.nonzero(np.isin(t, nbr))[0]
    I, J = np.meshgrid(cen, nb, indexing="ij")
    I, J = I.ravel(), J.ravel()
    keep = I != J
    I, J = I[keep], J[keep]
    dist = np.sqrt(((x[I] - x[J]) ** 2).sum(1))
    return I, J, dist


def test_sigma_to_zero_is_exact_histogram(orc, spec):
    xyz, t, d = _cloud(spec, 41, 40, 2.0)
    r0, dr, nb = 0.0, 0.1, 20
    _, _, dist = _pairs(xyz, t, d, [0, 1], [0, 1], 0.0)
    e = r0 + np.arange(nb + 1) * dr
    gap = np.min(np.abs(dist[:, None] - e[None, :]))
    assert gap > 1e-5  # no pair within float32 rounding of an edge
    sigma = gap / 40.0
    h = orc.soft_fwd(xyz, t, d, [0, 1], [0, 1], 0.0, sigma, 1.0, r0, dr, nb)
    H = orc.spatstat(xyz, t, d, [0, 1], [0, 1], 0.0, r0, dr, nb)["rdf"].astype(np.float64)
    np.testing.assert_array_equal(h, H)


def test_telescoping_sum(orc, spec):
    xyz, t, d = _cloud(spec, 42, 300, 3.5)
    for scale in (1.0, 0.93):
        h = orc.soft_fwd(xyz, t, d, [1], [0, 1], 0.5, SIG, scale, R0, DR, NB)
        _, _, dist = _pairs(xyz, t, d, [1], [0, 1], 0.5)
        u = scale * dist
        u = u[u < R0 + NB * DR + 6 * SIG]
        stop = R0 + NB * DR
        expect = np.sum(ndtr((stop - u) / SIG) - ndtr((R0 - u) / SIG))
        assert abs(h.sum() - expect) <= 1e-9 * expect


def _loss(orc, xyz, t, d, G, scale):
    return float(G @ orc.soft_fwd(xyz, t, d, "all", "all", 0.3, SIG, scale, R0, DR, NB))


def test_adjoint_matches_central_finite_differences(orc, spec):
    xyz, t, d = _cloud(spec, 43, 250, 3.4)
    xyz = xyz + np.float32(4.0)  # coordinates in [4, 8): steps of 2^-13 are exact in float32
    G = np.random.default_rng(5).standard_normal(NB)
    scale = 1.0
    gx, gs = orc.soft_bwd(xyz, t, d, "all", "all", 0.3, SIG, scale, R0, DR, NB, G)
    eps = 2.0**-13
    rng = np.random.default_rng(6)
    gmax = np.abs(gx).max()
    assert gmax > 0
    for i in rng.choice(xyz.shape[0], 12, replace=False):
        for a in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[i, a] += np.float32(eps)
            xm[i, a] -= np.float32(eps)
            assert float(xp[i, a]) - float(xm[i, a]) == 2 * eps
            fd = (_loss(orc, xp, t, d, G, scale) - _loss(orc, xm, t, d, G, scale)) / (2 * eps)
            assert abs(fd - gx[i, a]) <= 1e-6 * gmax, (i, a, fd, gx[i, a])
    es = 1e-5
    fds = (_loss(orc, xyz, t, d, G, scale + es) - _loss(orc, xyz, t, d, G, scale - es)) / (2 * es)
    assert abs(fds - gs) <= 1e-6 * max(abs(gs), 1.0)


def test_translation_and_scaling_identities(orc, spec):
    xyz, t, d = _cloud(spec, 44, 300, 3.5)
    G = np.random.default_rng(7).standard_normal(NB)
    for scale in (1.0, 1.07):
        gx, gs = orc.soft_bwd(xyz, t, d, [0], [0, 1], 0.2, SIG, scale, R0, DR, NB, G)
        tot = np.abs(gx).sum()
        assert np.all(np.abs(gx.sum(0)) <= 1e-12 * tot)
        euler = float((xyz.astype(np.float64) * gx).sum())
        assert abs(scale * gs - euler) <= 1e-10 * tot * 10
