"""GPU parity of the Gaussian-smoothed RDF and its adjoint against the FP64 oracle.

Tolerances (float32 arithmetic, fine-grid second-order expansion):
  forward   ||h_gpu - h_ref|| <= 1e-5 ||h_ref||  and  |h_gpu - h_ref| <= 1e-5 max|h_ref| per bin
  adjoint   ||g_gpu - g_ref|| <= 1e-4 ||g_ref||, per component <= 1e-4 max|g_ref|, dL/ds within 1e-4
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIG = 0.05
BINS = (0.0, 0.02, 100)


@pytest.fixture(scope="module")
def ps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2004_05188_gb300 as ps

    return ps


def _dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


def _run(ps, xyz, t, d, nbr, ctr, dmin, scale, G, cell_scale=1.0):
    X, T, D = _dev(xyz, t, d)
    g = ps.Grid(X.shape[0], cell_scale).build(X, T, nbr, ps.soft_r_cut(BINS, SIG, scale))
    h = ps.soft_rdf_fwd(g, D, ctr, dmin, SIG, scale, BINS)
    Gt = torch.from_numpy(G.astype(np.float32)).cuda()
    gx, gs = ps.soft_rdf_bwd(g, D, ctr, dmin, SIG, scale, BINS, Gt)
    torch.cuda.synchronize()
    assert g.info()["status"] == 0
    out = h.cpu().numpy().astype(np.float64), gx.cpu().numpy().astype(np.float64), float(gs.cpu()[0])
    g.close()
    return out


def _check(orc, xyz, t, d, nbr, ctr, dmin, scale, G, h, gx, gs):
    href = orc.soft_fwd(xyz, t, d, ctr, nbr, dmin, SIG, scale, *BINS)
    gref, gsref = orc.soft_bwd(xyz, t, d, ctr, nbr, dmin, SIG, scale, *BINS, G)
    assert np.linalg.norm(h - href) <= 1e-5 * np.linalg.norm(href)
    assert np.max(np.abs(h - href)) <= 1e-5 * np.max(np.abs(href))
    assert np.linalg.norm(gx - gref) <= 1e-4 * np.linalg.norm(gref)
    assert np.max(np.abs(gx - gref)) <= 1e-4 * np.max(np.abs(gref))
    assert abs(gs - gsref) <= 1e-4 * abs(gsref)
    return href, gref, gsref


@pytest.mark.parametrize("scale,cell_scale", [(1.0, 1.0), (0.93, 1.0), (1.07, 0.5), (1.0, 1 / 3)])
def test_soft_forward_and_adjoint_vs_fp64(ps, orc, spec, scale, cell_scale):
    xyz, t, d = spec.cube(201, 1500, 3.7, (0.7, 0.3))
    G = np.random.default_rng(11).standard_normal(BINS[2])
    h, gx, gs = _run(ps, xyz, t, d, "all", "all", 0.0, scale, G, cell_scale)
    _check(orc, xyz, t, d, "all", "all", 0.0, scale, G, h, gx, gs)


def test_soft_type_subsets_and_dsrf(ps, orc, spec):
    xyz, t, d = spec.cube(202, 2000, 4.0, (0.6, 0.3, 0.1))
    G = np.random.default_rng(12).standard_normal(BINS[2])
    h, gx, gs = _run(ps, xyz, t, d, [0, 2], [1], 0.6, 1.0, G)
    href, gref, _ = _check(orc, xyz, t, d, [0, 2], [1], 0.6, 1.0, G, h, gx, gs)
    # ions in no pair have exactly zero gradient (non-central ions of type 1 are not neighbours)
    cen = (t == 1) & (d >= 0.6)
    lonely = (t == 1) & ~cen
    assert np.all(gx[lonely] == 0.0)


@pytest.mark.parametrize("cell_scale", [1.0, 0.5])
def test_soft_centrals_within_neighbours(ps, orc, spec, cell_scale):
    """Centrals a subset of the neighbour set (one adjoint pass, pair weights 0, 1 and 2): type 1
    ions with d_srf >= 0.6 among neighbours of types {0, 1}; type 2 ions are in no pair."""
    xyz, t, d = spec.cube(204, 2000, 4.0, (0.5, 0.3, 0.2))
    G = np.random.default_rng(16).standard_normal(BINS[2])
    h, gx, gs = _run(ps, xyz, t, d, [0, 1], [1], 0.6, 0.97, G, cell_scale)
    _check(orc, xyz, t, d, [0, 1], [1], 0.6, 0.97, G, h, gx, gs)
    assert np.all(gx[t == 2] == 0.0)


def test_soft_identities_at_scale(ps, spec):
    """Translation invariance and the scaling identity on a 2e5-ion cylinder (any size)."""
    xyz, t, d = spec.cylinder_small()
    G = np.random.default_rng(13).standard_normal(BINS[2])
    h, gx, gs = _run(ps, xyz, t, d, "all", "all", 2.3, 1.0, G)
    tot = np.abs(gx).sum()
    assert np.all(np.abs(gx.sum(0)) <= 1e-4 * tot)
    euler = float((xyz.astype(np.float64) * gx).sum())
    assert abs(gs - euler) <= 1e-4 * abs(gs)
    assert h.min() >= 0 and h.sum() > 0


def test_autograd_function_matches_oracle(ps, orc, spec):
    xyz, t, d = spec.cube(203, 1200, 3.4, (1.0,))
    X = torch.from_numpy(xyz).cuda().requires_grad_(True)
    T, D = _dev(t, d)
    s = torch.tensor(1.02, dtype=torch.float32, device="cuda", requires_grad=True)
    target = torch.linspace(0, 1, BINS[2], device="cuda")
    h = ps.soft_rdf(X, s, T, D, "all", "all", 0.0, SIG, BINS)
    loss = ((h / h.sum() - target / target.sum()) ** 2).sum()
    loss.backward()
    # the upstream gradient dL/dh, computed by torch on the same h
    hh = h.detach().clone().requires_grad_(True)
    l2 = ((hh / hh.sum() - target / target.sum()) ** 2).sum()
    (Gh,) = torch.autograd.grad(l2, [hh])
    gref, gsref = orc.soft_bwd(xyz, t, d, "all", "all", 0.0, SIG, 1.02, *BINS, Gh.cpu().numpy().astype(np.float64))
    gx = X.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gx - gref) <= 1e-4 * np.linalg.norm(gref)
    assert abs(float(s.grad) - gsref) <= 1e-4 * abs(gsref)


def test_soft_gradient_vs_fp64_finite_differences_on_needle_subset(ps, orc, spec):
    """2,000 ions of the 1e7-ion needle (the ions nearest the axis in a 3.6 nm slab at mid height):
    the GPU adjoint against FP64 central differences of the oracle forward."""
    p = spec.needle_10m_params()
    counts = spec.needle_plan(p)
    k0 = counts.shape[0] // 2
    n = int(counts[k0:k0 + 9].sum())
    xyz = np.empty((n, 3), np.float32)
    t = np.empty(n, np.uint8)
    d = np.empty(n, np.float32)
    spec.needle_fill(p, k0, k0 + 9, counts, xyz.ctypes.data, t.ctypes.data, d.ctypes.data)
    sel = np.sort(np.argsort(np.hypot(xyz[:, 0], xyz[:, 1]))[:2000])
    xyz, t, d = xyz[sel], t[sel], d[sel]
    d = np.full_like(d, 10.0)  # every ion of the subset is central
    G = np.random.default_rng(14).standard_normal(BINS[2])
    h, gx, gs = _run(ps, xyz, t, d, "all", "all", 0.0, 1.0, G)
    gref, gsref = orc.soft_bwd(xyz, t, d, "all", "all", 0.0, SIG, 1.0, *BINS, G)
    assert np.linalg.norm(gx - gref) <= 1e-4 * np.linalg.norm(gref)

    def loss(x, s=1.0):
        return float(G @ orc.soft_fwd(x, t, d, "all", "all", 0.0, SIG, s, *BINS))

    eps = 2.0**-13  # |x|, |y| < 4 nm here: x +- eps is exact in float32
    gmax = np.abs(gref).max()
    for i, a in [(17, 0), (1000, 1), (1999, 0)]:
        assert abs(xyz[i, a]) < 4.0
        xp, xm = xyz.copy(), xyz.copy()
        xp[i, a] += np.float32(eps)
        xm[i, a] -= np.float32(eps)
        fd = (loss(xp) - loss(xm)) / (2 * eps)
        assert abs(gx[i, a] - fd) <= 1e-4 * gmax, (i, a, gx[i, a], fd)
    es = 1e-5
    fds = (loss(xyz, 1 + es) - loss(xyz, 1 - es)) / (2 * es)
    assert abs(gs - fds) <= 1e-4 * abs(fds)


def test_soft_identities_on_1e7_needle(ps, spec):
    """The full 1e7-ion needle of the smoothed-RDF workload: translation invariance and the scaling
    identity of the adjoint, and h >= 0 summing to about the exact in-range pair count."""
    xyz, t, d = spec.needle(spec.needle_10m_params())
    G = np.random.default_rng(15).standard_normal(BINS[2])
    h, gx, gs = _run(ps, xyz, t, d, "all", "all", 2.3, 1.0, G)
    tot = np.abs(gx).sum()
    assert np.all(np.abs(gx.sum(0)) <= 1e-4 * tot)
    # Euler: s dL/ds = sum_i x_i . dL/dx_i, about the centroid (the same identity, since the
    # gradients sum to zero; it keeps the float32 gradients' residual sum out of the comparison)
    xc = xyz.astype(np.float64) - xyz.astype(np.float64).mean(axis=0)
    euler = float((xc * gx).sum())
    assert abs(gs - euler) <= 1e-4 * abs(gs)
    X, T, D = _dev(xyz, t, d)
    g = ps.Grid(X.shape[0]).build(X, T, "all", 2.0)
    o = ps.spatstat(g, D, "all", 2.3, BINS, [])
    n_pairs = int(o["meta"][1].item())
    assert h.min() >= 0 and abs(h.sum() - n_pairs) <= 2e-3 * n_pairs
    g.close()


def test_soft_1e7_needle_sampled_centrals_vs_fp64(ps, orc, spec):
    """The 1e7-ion needle at full size: 2,000 centrals drawn from a 1 nm z-slab at mid-height (every
    other ion's d_srf set to NaN, so no other ion is central), forward and adjoint on the grid of
    the whole cloud, against the FP64 oracle on those centrals with every ion within reach of them
    (the slab +- 3 nm), the centrals split over the host cores (h and the gradients are sums over
    pairs, so the parts add up).  Ions outside the oracle's sub-cloud are in no pair: their GPU
    gradient must be exactly zero."""
    import concurrent.futures as cf
    import os

    xyz, t, d = spec.needle(spec.needle_10m_params())
    z = xyz[:, 2]
    z0 = float(np.median(z))
    slab = np.nonzero((z >= z0) & (z < z0 + 1.0) & (d >= np.float32(2.3)))[0]
    rng = np.random.default_rng(16)
    cen = np.sort(rng.choice(slab, 2000, replace=False))
    dm = np.full_like(d, np.float32(np.nan))
    dm[cen] = d[cen]
    G = rng.standard_normal(BINS[2])
    h, gx, gs = _run(ps, xyz, t, dm, "all", "all", 2.3, 1.0, G)
    sub = np.nonzero((z >= z0 - 3.0) & (z < z0 + 4.0))[0]
    assert np.all(gx[np.setdiff1d(np.arange(xyz.shape[0]), sub)] == 0.0)
    xs, ts = xyz[sub], t[sub]
    pos = np.searchsorted(sub, cen)
    threads = min(16, os.cpu_count() or 8)

    def part(k):
        dk = np.full(sub.shape[0], np.float32(np.nan), np.float32)
        mine = pos[k::threads]
        dk[mine] = dm[cen[k::threads]]
        hk = orc.soft_fwd(xs, ts, dk, "all", "all", 2.3, SIG, 1.0, *BINS)
        gk, gsk = orc.soft_bwd(xs, ts, dk, "all", "all", 2.3, SIG, 1.0, *BINS, G)
        return hk, gk, gsk

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(part, range(threads)))
    href = sum(p[0] for p in parts)
    gref = sum(p[1] for p in parts)
    gsref = sum(p[2] for p in parts)
    assert np.linalg.norm(h - href) <= 1e-5 * np.linalg.norm(href)
    assert np.max(np.abs(h - href)) <= 1e-5 * np.max(np.abs(href))
    gxs = gx[sub]
    assert np.linalg.norm(gxs - gref) <= 1e-4 * np.linalg.norm(gref)
    assert np.max(np.abs(gxs - gref)) <= 1e-4 * np.max(np.abs(gref))
    assert abs(gs - gsref) <= 1e-4 * abs(gsref)
