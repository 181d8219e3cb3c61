"""GPU parity of the spatial distribution map (ps_sdm) against the oracle: every voxel and every
counter bit-exact, on Poisson clouds, a precipitate needle, a simple-cubic lattice whose
displacements sit on voxel edges, a voxel cube smaller than the ROI, the grid options, the
degenerate cases and the argument checks."""
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


def _gpu_sdm(ps, xyz, t, d, ctr, nbr, dmin, R, w, nv, cell_scale=1.0, dense_min=0, r_cut=None):
    X, T, D = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (xyz, t, d))
    g = ps.Grid(X.shape[0], cell_scale, dense_min).build(X, T, nbr, r_cut or R * (1 + 1e-6))
    out = ps.sdm(g, D, ctr, dmin, R, w, nv)
    torch.cuda.synchronize()
    H, meta = out["H"].cpu().numpy(), out["meta"].cpu().numpy()
    g.close()
    return H, meta


def _same(ps, orc, xyz, t, d, ctr, nbr, dmin, R, w, nv, **kw):
    H, meta = _gpu_sdm(ps, xyz, t, d, ctr, nbr, dmin, R, w, nv, **kw)
    Ho, mo = orc.sdm(xyz, t, d, ctr, nbr, dmin, R, w, nv)
    assert meta[3] == 0, f"device status {meta[3]}"
    np.testing.assert_array_equal(meta[:3].astype(np.uint64), mo)
    np.testing.assert_array_equal(H.astype(np.uint64), Ho)
    return H, meta


@pytest.mark.parametrize("ctr,nbr,dmin", [("all", "all", 1.0), ([1], [1], 0.5), ([0], [1, 2], 1.5), ([2], "all", -1.0)])
def test_sdm_poisson_cylinder(ps, orc, spec, ctr, nbr, dmin):
    xyz, t, d = spec.cylinder(7, 20000, 6.0, 8.0, (0.6, 0.3, 0.1))
    H, meta = _same(ps, orc, xyz, t, d, ctr, nbr, dmin, 2.0, 0.025, 160)
    assert meta[1] > 0


def test_sdm_needle_sc_sc_and_al_sc(ps, orc, spec):
    xyz, t, d = spec.needle(spec.needle_params(r_top=8.0, half_angle_deg=10.0, height=20.0, seed=9))
    for ctr, nbr in (([1], [1]), ([0], [1])):
        _same(ps, orc, xyz, t, d, ctr, nbr, 2.0, 2.0, 0.025, 160)


def test_sdm_lattice_on_voxel_edges(ps, orc, spec):
    xyz, t, d = spec.simple_cubic(24)
    H, meta = _same(ps, orc, xyz, t, d, [0], [0], 2.0, 2.0, 0.025, 160)
    n_c = int(meta[0])
    assert n_c > 0 and H[80, 80, 90] == n_c and H[80, 80, 89] == 0


@pytest.mark.parametrize("cell_scale,dense_min", [(0.5, 0), (1.0, 16), (0.75, 64)])
def test_sdm_grid_options(ps, orc, spec, cell_scale, dense_min):
    xyz, t, d = spec.cylinder(8, 20000, 6.0, 8.0, (0.7, 0.3))
    _same(ps, orc, xyz, t, d, "all", "all", 1.0, 1.5, 0.05, 60, cell_scale=cell_scale, dense_min=dense_min)


def test_sdm_cube_smaller_than_roi(ps, orc, spec):
    xyz, t, d = spec.cylinder(9, 8000, 5.0, 6.0, (1.0,))
    H, meta = _same(ps, orc, xyz, t, d, "all", "all", 0.0, 2.0, 0.05, 33)
    assert meta[2] > 0


def test_sdm_empty_and_single(ps, orc, spec):
    xyz, t, d = spec.cylinder(10, 3000, 4.0, 5.0, (1.0,))
    H, meta = _same(ps, orc, xyz, t, d, [5], "all", 0.0, 1.0, 0.1, 20)  # no central of type 5
    assert meta[0] == 0 and H.sum() == 0
    _same(ps, orc, xyz[:1], t[:1], d[:1], "all", "all", 0.0, 1.0, 0.1, 20)


def test_sdm_argument_checks(ps, spec):
    xyz, t, d = spec.cylinder(11, 1000, 3.0, 3.0, (1.0,))
    X, T, D = (torch.from_numpy(a).cuda() for a in (xyz, t, d))
    g = ps.Grid(1000).build(X, T, "all", 1.0)
    with pytest.raises(RuntimeError):
        ps.sdm(g, D, "all", 0.0, 1.5, 0.05, 60)  # r_max above the grid's r_cut
    with pytest.raises(RuntimeError):
        ps.sdm(g, D, "all", 0.0, 1.0, 0.05, 0)
    with pytest.raises(RuntimeError):
        ps.sdm(g, D, "all", 0.0, 1.0, -0.05, 10)
    g.close()
