"""Host check of the near kNN pass's geometric guarantee (the query in passes on half-size cells):
every record outside the 2 x 2 x 2 cells around a central's vertex lies at a squared distance of
at least the central's reach.  The cell coordinates, the vertex-centred cells and the reach are
restated here with float32 numpy arithmetic in the kernel's operation order (cell coordinate
u = (x - origin) * inv_h; vertex cell from the origin half a cell lower; reach = (distance to the
block's faces - slack) * h * (1 - 2^-12), squared, times (1 - 2^-12)), and checked by brute force
on random clouds with points placed on and next to the cell faces."""
import numpy as np
import pytest

f32 = np.float32


def _grid(xyz, r_cut, cell_scale):
    lo = xyz.min(axis=0).astype(np.float64)
    hi = xyz.max(axis=0).astype(np.float64)
    ext = float((hi - lo).max())
    h = r_cut * cell_scale * (1.0 + 1.0 / 1024.0) + ext / 1048576.0
    dims = np.floor((hi - lo) / h).astype(np.int64) + 1
    org = lo.astype(np.float32)
    hf = f32(h)
    inv_h = f32(1.0 / h)
    return org, hf, inv_h, dims


def _cells(P, org, inv_h, dims):
    u = (P - org).astype(f32) * inv_h  # two float32 roundings, as the kernel
    c = np.floor(u).astype(np.int64)
    return np.clip(c, 0, dims - 1), u


@pytest.mark.parametrize("seed,n,box", [(1, 3000, 9.0), (2, 2500, 14.0), (3, 2000, 6.0)])
def test_vertex_reach_bounds_every_record_outside_the_block(seed, n, box):
    rng = np.random.default_rng(seed)
    r_cut, cs = 2.0, 0.5
    xyz = (rng.random((n, 3)) * box).astype(f32)
    org, hf, inv_h, dims = _grid(xyz, r_cut, cs)
    # points on, just below and just above the cell faces and the midplanes (the vertex cell's
    # faces), where the rounding of the coordinates decides the cells
    k = rng.integers(0, dims.min(), size=(n // 2, 3))
    frac = rng.choice([0.0, 0.5, 1.0], size=(n // 2, 3))
    eps = rng.choice([-1, 0, 1], size=(n // 2, 3)) * 2.0 ** -22 * box
    face = (org.astype(np.float64) + (k + frac) / np.float64(inv_h) + eps).astype(f32)
    xyz = np.concatenate([xyz, face])
    org, hf, inv_h, dims = _grid(xyz, r_cut, cs)
    c, u = _cells(xyz, org, inv_h, dims)
    # vertex-centred cells: origin half a cell lower, one more cell per axis
    org_v = (org - f32(f32(0.5) * hf)).astype(f32)
    V, _ = _cells(xyz, org_v, inv_h, dims + 1)
    # reach (kernel order)
    slack = f32(float(dims.max()) * 5.0e-7 + 1.0e-6)
    h_eff = f32(f32(1.0) / inv_h) * f32(1.0 - 1.0 / 4096.0)
    m = np.minimum(u - (V.astype(f32) - f32(1.0)), (V.astype(f32) + f32(1.0)) - u).astype(f32).min(axis=1)
    r = (np.maximum(m - slack, f32(0.0)) * h_eff).astype(f32)
    e = ((r * r).astype(f32) * f32(1.0 - 1.0 / 4096.0)).astype(f32)
    assert np.all(m > 0.45)  # every central is about half a cell or more inside its block
    # brute force: records outside the block [V - 1, V] (neighbour-cell coordinates) per axis
    for i in range(xyz.shape[0]):
        outside = np.any((c < V[i] - 1) | (c > V[i]), axis=1)
        q = xyz[outside]
        dx, dy, dz = (q[:, 0] - xyz[i, 0]), (q[:, 1] - xyz[i, 1]), (q[:, 2] - xyz[i, 2])
        d2 = ((dx * dx + dy * dy).astype(f32) + (dz * dz)).astype(f32)
        assert d2.size == 0 or d2.min() >= e[i], (i, float(d2.min()), float(e[i]))


@pytest.mark.parametrize("cell_scale", [1 / 3, 0.4, 0.75, 0.6])
def test_skipped_cells_hold_no_pair_within_r_cut(cell_scale):
    """The stencil rows' widths (the cells a query skips because their gap to the central cell is
    at least r_cut on the cell-edge bound): every pair with float32 d2 below r_cut^2 lies in a
    kept cell offset, by brute force over a dense random cloud with points on the cell faces."""
    import bench

    rng = np.random.default_rng(11)
    r_cut = 2.0
    xyz = (rng.random((2500, 3)) * 7.0).astype(f32)
    org, hf, inv_h, dims = _grid(xyz, r_cut, cell_scale)
    k = rng.integers(0, dims.min(), size=(1500, 3))
    face = (org.astype(np.float64) + k / np.float64(inv_h)
            + rng.choice([-1, 0, 1], size=(1500, 3)) * 2.0 ** -22 * 7.0).astype(f32)
    xyz = np.concatenate([xyz, face])
    org, hf, inv_h, dims = _grid(xyz, r_cut, cell_scale)
    c, _ = _cells(xyz, org, inv_h, dims)
    s = 1 if cell_scale >= 1.0 else (2 if cell_scale >= 0.5 else 3)
    w = np.array(bench.row_widths(s, cell_scale))  # [dz + s][dy + s]
    E = f32(r_cut * r_cut)
    for i in range(xyz.shape[0]):
        dx, dy, dz = (xyz[:, 0] - xyz[i, 0]), (xyz[:, 1] - xyz[i, 1]), (xyz[:, 2] - xyz[i, 2])
        d2 = ((dx * dx + dy * dy).astype(f32) + (dz * dz)).astype(f32)
        near = d2 < E
        off = c[near] - c[i]
        assert np.all(np.abs(off) <= s), i
        width = w[off[:, 2] + s, off[:, 1] + s]
        assert np.all(np.abs(off[:, 0]) <= width), (i, off[np.abs(off[:, 0]) > width][:3])


def test_first_tier_reach_of_the_full_radius_pass():
    """The full-radius pass settles a central after the 27 cells around its cell when its k-th
    distance lies within its reach to the faces of that block (cells c - 1 .. c + 1): no record
    outside those cells lies below the reach."""
    rng = np.random.default_rng(5)
    r_cut, cs = 2.0, 0.5
    xyz = (rng.random((2500, 3)) * 10.0).astype(f32)
    org, hf, inv_h, dims = _grid(xyz, r_cut, cs)
    k = rng.integers(0, dims.min(), size=(1500, 3))
    face = (org.astype(np.float64) + k / np.float64(inv_h)
            + rng.choice([-1, 0, 1], size=(1500, 3)) * 2.0 ** -22 * 10.0).astype(f32)
    xyz = np.concatenate([xyz, face])
    org, hf, inv_h, dims = _grid(xyz, r_cut, cs)
    c, u = _cells(xyz, org, inv_h, dims)
    slack = f32(float(dims.max()) * 5.0e-7 + 1.0e-6)
    h_eff = f32(f32(1.0) / inv_h) * f32(1.0 - 1.0 / 4096.0)
    m = np.minimum(u - (c.astype(f32) - f32(1.0)), (c.astype(f32) + f32(2.0)) - u).astype(f32).min(axis=1)
    r = (np.maximum(m - slack, f32(0.0)) * h_eff).astype(f32)
    e = ((r * r).astype(f32) * f32(1.0 - 1.0 / 4096.0)).astype(f32)
    for i in range(xyz.shape[0]):
        outside = np.any(np.abs(c - c[i]) > 1, axis=1)
        q = xyz[outside]
        dx, dy, dz = (q[:, 0] - xyz[i, 0]), (q[:, 1] - xyz[i, 1]), (q[:, 2] - xyz[i, 2])
        d2 = ((dx * dx + dy * dy).astype(f32) + (dz * dz)).astype(f32)
        assert d2.size == 0 or d2.min() >= e[i], (i, float(d2.min()), float(e[i]))
