"""GB300-native spatial statistics (exact kNN / RDF) for atom-probe point clouds.

Thin Python binding over the C ABI of libps (include/ps.h): argument
marshalling only.  Every step of the computation runs in the CUDA kernels of
libps.so; there is no CPU fallback.  PyTorch supplies device memory and
streams.  Importing this package works without a GPU (host helpers only);
calling a compute function without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libps.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "ps.h")

PS_OK = 0
STATIC_MAX_IONS = 262144
STATUS = {0: "PS_OK", 1: "PS_ERR_INVALID_ARG", 2: "PS_ERR_INVALID_INPUT", 3: "PS_ERR_OOM", 4: "PS_ERR_CUDA",
          5: "PS_ERR_TIMEOUT", 6: "PS_ERR_UNSUPPORTED", 7: "PS_ERR_CAPACITY"}
K_MAX = 32
MAX_BINS = 8192
MAX_KLIST = 32
META_HEAD = 4
AL, SC, SI = 0, 1, 2


class PSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def bins_from_spec(start: float, step: float, stop: float):
    """The paper's bin notation r = [start, step, stop] (nm) -> (r0, dr, n_bins).

    n_bins = round((stop - start) / step) in double; r0 and dr stay double so
    that edges such as 0.25 nm on a 0.01 nm step are exact.
    """
    if not (step > 0) or not (stop > start) or start < 0:
        raise ValueError("need 0 <= start < stop and step > 0")
    return float(start), float(step), int(round((stop - start) / step))


def type_mask(types) -> np.ndarray:
    """Type set -> 4 x uint64 bit mask; `types` is an iterable of labels or 'all'."""
    m = np.zeros(4, dtype=np.uint64)
    if isinstance(types, str):
        if types != "all":
            raise ValueError("type set must be an iterable of labels or 'all'")
        m[:] = np.uint64(0xFFFFFFFFFFFFFFFF)
        return m
    for t in types:
        t = int(t)
        if not 0 <= t < 256:
            raise ValueError("type labels are 0..255")
        m[t >> 6] |= np.uint64(1) << np.uint64(t & 63)
    return m


class Bins(ctypes.Structure):
    _fields_ = [("r0", ctypes.c_double), ("dr", ctypes.c_double), ("n_bins", ctypes.c_uint32)]


class GridOpts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("cell_scale", ctypes.c_float), ("block", ctypes.c_uint32),
                ("dense_min", ctypes.c_uint32), ("split", ctypes.c_uint32)]


class GridInfo(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("dims", ctypes.c_uint32 * 3), ("origin", ctypes.c_float * 3),
                ("cell", ctypes.c_float), ("n_nbr", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("status", ctypes.c_int32)]


class Dataset(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_void_p), ("type", ctypes.c_void_p), ("dsrf", ctypes.c_void_p), ("n", ctypes.c_int64)]


class SdmSpec(ctypes.Structure):
    _fields_ = [("r_max", ctypes.c_double), ("w", ctypes.c_double), ("n_vox", ctypes.c_uint32)]


class ClusterSpec(ctypes.Structure):
    _fields_ = [("d_max", ctypes.c_double), ("n_min", ctypes.c_uint32), ("dsrf_min", ctypes.c_float),
                ("hist_len", ctypes.c_uint32)]


class Sweep(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("bins", Bins), ("n_rmax", ctypes.c_uint32),
                ("rmax_bins", ctypes.c_uint32 * 4), ("n_dsrf", ctypes.c_uint32), ("dsrf_min", ctypes.c_float * 4),
                ("n_pairs", ctypes.c_uint32), ("ctr_mask", (ctypes.c_uint64 * 4) * 4),
                ("nbr_mask", (ctypes.c_uint64 * 4) * 4), ("k_max", ctypes.c_uint32), ("cell_scale", ctypes.c_float)]


class Peaks(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("num_sms", ctypes.c_int32), ("fp32_scalar_gops", ctypes.c_double),
                ("fp32_packed_gops", ctypes.c_double), ("smem_atomic_gops", ctypes.c_double),
                ("sm_mhz", ctypes.c_double)]


_lib = None


def header_functions():
    """Names of the entry points declared in include/ps.h."""
    with open(HEADER) as f:
        txt = f.read()
    return sorted(set(re.findall(r"PS_API\s+[\w\s\*]+?\b(ps_\w+)\s*\(", txt)))


def lib():
    """Load libps.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libps.so not built ({LIB_PATH}); run __graft_entry__.build() first")
    L = ctypes.CDLL(LIB_PATH)
    P, i64, u32, f32, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float, ctypes.c_int
    L.ps_version.restype = i32
    L.ps_last_error.restype = ctypes.c_char_p
    L.ps_bin_edges.argtypes = [Bins, P]
    L.ps_grid_create.argtypes = [i64, ctypes.POINTER(GridOpts), ctypes.POINTER(P)]
    L.ps_grid_build.argtypes = [P, P, P, i64, P, f32, P]
    L.ps_build_grid.argtypes = [P, P, i64, P, f32, ctypes.POINTER(GridOpts), P, ctypes.POINTER(P)]
    L.ps_grid_destroy.argtypes = [P]
    L.ps_grid_set_query_opts.argtypes = [P, u32, u32]
    L.ps_grid_get_info.argtypes = [P, ctypes.POINTER(GridInfo), P]
    L.ps_spatstat.argtypes = [P, P, P, f32, Bins, P, u32, P, P, P, P, P, P]
    L.ps_knn_hist.argtypes = [P, P, P, f32, u32, Bins, P, P, P, P]
    L.ps_rdf_hist.argtypes = [P, P, P, f32, Bins, P, P, P]
    L.ps_batch_create.argtypes = [ctypes.POINTER(Dataset), ctypes.c_int, ctypes.POINTER(Sweep), ctypes.POINTER(P)]
    L.ps_batch_run.argtypes = [P, P, P]
    L.ps_batch_out_len.argtypes = [P]
    L.ps_batch_out_len.restype = ctypes.c_int64
    L.ps_batch_destroy.argtypes = [P]
    L.ps_rdf_soft_fwd.argtypes = [P, P, P, f32, f32, f32, Bins, P, P]
    L.ps_rdf_soft_bwd.argtypes = [P, P, P, f32, f32, f32, Bins, P, P, P, P]
    L.ps_shuffle_labels.argtypes = [P, P, i64, ctypes.c_uint64, P, P]
    L.ps_sdm.argtypes = [P, P, P, f32, SdmSpec, P, P, P]
    L.ps_cluster.argtypes = [P, P, ClusterSpec, P, P, P, P, P]
    L.ps_spatstat_static.argtypes = [P, P, P, i64, P, f32, P, f32, Bins, P, u32, P, P, P, P, P, P]
    L.ps_rdf_normalise.argtypes = [P, P, P, ctypes.c_double, Bins, P, P, P]
    L.ps_measure_peaks.argtypes = [ctypes.POINTER(Peaks), P]
    L.ps_debug_fail_alloc.argtypes = [i64]
    L.ps_debug_live_allocs.restype = i64
    L.ps_debug_wait_selftest.argtypes = [ctypes.c_uint64, P, P]
    L.ps_launch_count.restype = ctypes.c_uint64
    L.ps_prof_enable.argtypes = [u32]
    L.ps_prof_read.argtypes = [u32, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]
    _lib = L
    return L


def _check(rc: int):
    if rc != PS_OK:
        raise PSError(rc, lib().ps_last_error().decode(errors="replace"))


KID = dict(reset=1, select=2, geometry=3, count=4, scan=5, scatter=6, central=7, query=8, epilogue=9, soft_fwd=10,
           soft_bwd=11, batch=12, labels=13, sdm=14, cluster=15, finalise=16, peaks=17, rdf_sym=18, knn_full=19)


def measure_peaks(stream=None) -> dict:
    """Measured FP32 add/multiply, shared-atomic throughput and SM clock of the current GPU
    (ps_measure_peaks; synchronises)."""
    p = Peaks()
    p.struct_size = ctypes.sizeof(Peaks)
    _check(lib().ps_measure_peaks(ctypes.byref(p), _stream(stream)))
    return dict(num_sms=p.num_sms, fp32_scalar_gops=p.fp32_scalar_gops, fp32_packed_gops=p.fp32_packed_gops,
                smem_atomic_gops=p.smem_atomic_gops, sm_mhz=p.sm_mhz)


def launch_count() -> int:
    """Kernels launched by libps in this process."""
    return int(lib().ps_launch_count())


def prof_enable(kernels=()) -> None:
    """Time every launch of the named kernel families with CUDA events (resets the tallies)."""
    mask = 0
    for k in kernels:
        mask |= 1 << KID[k]
    _check(lib().ps_prof_enable(mask))


def prof_read(kernel: str):
    """(launches, total ms) of one kernel family since prof_enable."""
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(lib().ps_prof_read(KID[kernel], ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def edges(r0: float, dr: float, n_bins: int) -> np.ndarray:
    """The float32 edge table E[0..n_bins] of libps (host computation)."""
    E = np.empty(n_bins + 1, np.float32)
    _check(lib().ps_bin_edges(Bins(r0, dr, n_bins), E.ctypes.data_as(ctypes.c_void_p)))
    return E


def _stream(stream):
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _mask_ptr(types):
    m = type_mask(types)
    return m, m.ctypes.data_as(ctypes.c_void_p)


def _check_cloud(xyz, type_, dsrf=None):
    import torch

    if not (xyz.is_cuda and type_.is_cuda):
        raise ValueError("xyz and type must be CUDA tensors")
    if xyz.dtype != torch.float32 or type_.dtype != torch.uint8:
        raise ValueError("xyz must be float32 and type uint8")
    if xyz.dim() != 2 or xyz.shape[1] != 3 or not xyz.is_contiguous() or not type_.is_contiguous():
        raise ValueError("xyz must be a contiguous [n, 3] tensor and type contiguous [n]")
    if type_.shape[0] != xyz.shape[0]:
        raise ValueError("xyz and type lengths differ")
    if dsrf is not None:
        if not dsrf.is_cuda or dsrf.dtype != torch.float32 or not dsrf.is_contiguous() or dsrf.shape[0] != xyz.shape[0]:
            raise ValueError("dsrf must be a contiguous float32 CUDA tensor of length n")


class Grid:
    """A cell grid over the neighbour set of one cloud (ps_grid_create / ps_grid_build)."""

    def __init__(self, n_max: int, cell_scale: float = 1.0, dense_min: int = 0, split: bool = False):
        """cell_scale: cell edge / r_cut (>= 1: 27-cell search; [0.5, 1): 125-cell search; [1/3, 0.5): 343
        cells less the far corners that cannot hold a pair within r_cut).
        dense_min: cells with at least this many centrals use the shared-memory staged kernel (0: never).
        split: run the exact query in passes where it applies (near-radius kNN with a full-radius
        fallback, RDF over unordered pairs); same results (see ps_grid_opts.split)."""
        opts = GridOpts(ctypes.sizeof(GridOpts), float(cell_scale), 0, int(dense_min), int(bool(split)))
        h = ctypes.c_void_p()
        _check(lib().ps_grid_create(int(n_max), ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self.n_max = int(n_max)
        self.cell_scale = float(np.float32(cell_scale if cell_scale else 1.0))
        # cells searched around a cell along each axis (the library's rule)
        self.stencil = 1 if self.cell_scale >= 1.0 else (2 if self.cell_scale >= 0.5 else 3)
        self._refs = ()

    @property
    def handle(self):
        return self._h

    def build(self, xyz, type_, nbr_types, r_cut: float, stream=None):
        _check_cloud(xyz, type_)
        m, mp = _mask_ptr(nbr_types)
        _check(lib().ps_grid_build(self._h, _ptr(xyz), _ptr(type_), xyz.shape[0], mp, float(r_cut), _stream(stream)))
        self._refs = (xyz, type_)  # the grid reads these again in every query
        self.n = int(xyz.shape[0])
        self.r_cut = float(r_cut)
        return self

    def set_query_opts(self, dense_min: int = 0, split: bool = False):
        """Query options for the next queries on this grid (ps_grid_set_query_opts); the cell size stays."""
        _check(lib().ps_grid_set_query_opts(self._h, int(dense_min), int(bool(split))))
        return self

    def info(self, stream=None) -> dict:
        gi = GridInfo()
        gi.struct_size = ctypes.sizeof(GridInfo)
        _check(lib().ps_grid_get_info(self._h, ctypes.byref(gi), _stream(stream)))
        return dict(dims=tuple(gi.dims), origin=tuple(gi.origin), cell=gi.cell, n_nbr=gi.n_nbr,
                    n_cells=gi.n_cells, status=gi.status)

    def close(self):
        if self._h:
            _check(lib().ps_grid_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.ps_grid_destroy(self._h)
        except Exception:
            pass


def spatstat(grid: Grid, dsrf, ctr_types, dsrf_min: float, bins, ks=(), rdf: bool = True, per_central: bool = False,
             out=None, stream=None, check: bool = True):
    """Exact RDF + kNN histograms in one enumeration (ps_spatstat).

    bins = (r0, dr, n_bins).  Returns a dict of CUDA tensors: rdf [n_bins],
    knn [n_k, n_bins], meta [4 + 2 n_k] (n_central, pairs binned, pairs below
    r0, status, then per k: not found, below r0) and, with per_central,
    kth_d2 [n_k, n] and n_within [n] (central ions only; others hold -1 / NaN).
    With check=True the device status is read back (one synchronisation).
    """
    import torch

    r0, dr, nb = bins
    ks = [int(k) for k in ks]
    nk = len(ks)
    dev = grid._refs[0].device
    if dsrf is not None:
        _check_cloud(grid._refs[0], grid._refs[1], dsrf)
    if out is None:
        out = {}
        out["rdf"] = torch.empty(nb, dtype=torch.int64, device=dev) if rdf else None
        out["knn"] = torch.empty((nk, nb), dtype=torch.int64, device=dev) if nk else None
        out["meta"] = torch.empty(META_HEAD + 2 * nk, dtype=torch.int64, device=dev)
        if per_central:
            out["kth_d2"] = torch.full((nk, grid.n), float("nan"), dtype=torch.float32, device=dev) if nk else None
            if per_central != "kth":
                out["n_within"] = torch.full((grid.n,), -1, dtype=torch.int32, device=dev)
    ks_a = np.ascontiguousarray(ks, np.uint32)
    m, mp = _mask_ptr(ctr_types)
    _check(lib().ps_spatstat(grid.handle, _ptr(dsrf), mp, float(dsrf_min), Bins(r0, dr, nb),
                             ks_a.ctypes.data_as(ctypes.c_void_p), nk, _ptr(out.get("rdf")), _ptr(out.get("knn")),
                             _ptr(out["meta"]), _ptr(out.get("kth_d2")), _ptr(out.get("n_within")), _stream(stream)))
    if check:
        st = int(out["meta"][3].item())
        if st != 0:
            raise PSError(st, "device-side error reported in the meta status word")
    return out


def rdf_normalise(grid: Grid, meta, bins, volume: float, rdf=None, stream=None):
    """Normalised RDF (ps_rdf_normalise) of a histogram computed on `grid` (not rebuilt since).

    meta: the int64 meta tensor of that spatstat call; volume: specimen volume (nm^3).
    Returns (g, factor): float64 CUDA tensors [n_bins]; g is None when rdf is None.
    factor_b = 1 / (|C| (|N| / volume) 4/3 pi (e_{b+1}^3 - e_b^3)), so g = rdf * factor."""
    import torch

    r0, dr, nb = bins
    dev = grid._refs[0].device
    f = torch.empty(nb, dtype=torch.float64, device=dev)
    g = torch.empty(nb, dtype=torch.float64, device=dev) if rdf is not None else None
    _check(lib().ps_rdf_normalise(grid.handle, _ptr(meta), _ptr(rdf), float(volume), Bins(r0, dr, nb), _ptr(g),
                                  _ptr(f), _stream(stream)))
    return g, f


def knn_hist(grid: Grid, dsrf, ctr_types, dsrf_min: float, k: int, bins, stream=None):
    """kNN histogram for one k (ps_knn_hist): returns (hist [n_bins], meta [6])."""
    import torch

    r0, dr, nb = bins
    dev = grid._refs[0].device
    h = torch.empty(nb, dtype=torch.int64, device=dev)
    meta = torch.empty(META_HEAD + 2, dtype=torch.int64, device=dev)
    m, mp = _mask_ptr(ctr_types)
    _check(lib().ps_knn_hist(grid.handle, _ptr(dsrf), mp, float(dsrf_min), int(k), Bins(r0, dr, nb), _ptr(h),
                             _ptr(meta), None, _stream(stream)))
    return h, meta


def rdf_hist(grid: Grid, dsrf, ctr_types, dsrf_min: float, bins, stream=None):
    """RDF histogram (ps_rdf_hist): returns (hist [n_bins], meta [4])."""
    import torch

    r0, dr, nb = bins
    dev = grid._refs[0].device
    h = torch.empty(nb, dtype=torch.int64, device=dev)
    meta = torch.empty(META_HEAD, dtype=torch.int64, device=dev)
    m, mp = _mask_ptr(ctr_types)
    _check(lib().ps_rdf_hist(grid.handle, _ptr(dsrf), mp, float(dsrf_min), Bins(r0, dr, nb), _ptr(h), _ptr(meta),
                             _stream(stream)))
    return h, meta


SDM_META_LEN = 4


def sdm(grid: Grid, dsrf, ctr_types, dsrf_min: float, r_max: float, w: float, n_vox: int, out=None, stream=None):
    """Spatial distribution map (ps_sdm): returns {"H": int64 [n_vox, n_vox, n_vox] indexed [mz, my, mx],
    "meta": int64 [4] = n_central, pairs in the map, pairs outside the voxel cube, status}."""
    import torch

    dev = grid._refs[0].device
    if out is None:
        out = dict(H=torch.empty((n_vox, n_vox, n_vox), dtype=torch.int64, device=dev),
                   meta=torch.empty(SDM_META_LEN, dtype=torch.int64, device=dev))
    m, mp = _mask_ptr(ctr_types)
    _check(lib().ps_sdm(grid.handle, _ptr(dsrf), mp, float(dsrf_min), SdmSpec(float(r_max), float(w), int(n_vox)),
                        _ptr(out["H"]), _ptr(out["meta"]), _stream(stream)))
    return out


CLUSTER_META_LEN = 5


def cluster(grid: Grid, dsrf, d_max: float, n_min: int, dsrf_min: float = 0.0, hist_len: int = 1024, out=None,
            stream=None):
    """Maximum-separation clustering of the grid's set (ps_cluster).  Returns {"label": int32 [n]
    (smallest original index of the ion's cluster, -1 if none), "size_hist", "interior_hist":
    int64 [hist_len], "meta": int64 [5] = ions in the set, clusters, ions in clusters, interior
    clusters, status}."""
    import torch

    dev = grid._refs[0].device
    n = grid._refs[0].shape[0]
    if out is None:
        out = dict(label=torch.empty(n, dtype=torch.int32, device=dev),
                   size_hist=torch.empty(hist_len, dtype=torch.int64, device=dev),
                   interior_hist=torch.empty(hist_len, dtype=torch.int64, device=dev),
                   meta=torch.empty(CLUSTER_META_LEN, dtype=torch.int64, device=dev))
    spec = ClusterSpec(float(d_max), int(n_min), float(dsrf_min), int(hist_len))
    _check(lib().ps_cluster(grid.handle, _ptr(dsrf), spec, _ptr(out["label"]), _ptr(out["size_hist"]),
                            _ptr(out["interior_hist"]), _ptr(out["meta"]), _stream(stream)))
    return out


def soft_rdf_fwd(grid: Grid, dsrf, ctr_types, dsrf_min: float, sigma: float, scale: float, bins, out=None,
                 stream=None):
    """Gaussian-smoothed RDF h[n_bins] (float32 CUDA tensor), ps_rdf_soft_fwd."""
    import torch

    r0, dr, nb = bins
    h = out if out is not None else torch.empty(nb, dtype=torch.float32, device=grid._refs[0].device)
    m, mp = _mask_ptr(ctr_types)
    _check(lib().ps_rdf_soft_fwd(grid.handle, _ptr(dsrf), mp, float(dsrf_min), float(sigma), float(scale),
                                 Bins(r0, dr, nb), _ptr(h), _stream(stream)))
    return h


def soft_rdf_bwd(grid: Grid, dsrf, ctr_types, dsrf_min: float, sigma: float, scale: float, bins, dLdh,
                 grad_xyz=None, grad_scale=None, stream=None):
    """Adjoint of soft_rdf_fwd (ps_rdf_soft_bwd): returns (dL/dxyz [n, 3], dL/dscale [1])."""
    import torch

    r0, dr, nb = bins
    dev = grid._refs[0].device
    dLdh = dLdh.contiguous().to(dtype=torch.float32)
    gx = grad_xyz if grad_xyz is not None else torch.empty((grid.n, 3), dtype=torch.float32, device=dev)
    gs = grad_scale if grad_scale is not None else torch.empty(1, dtype=torch.float32, device=dev)
    m, mp = _mask_ptr(ctr_types)
    _check(lib().ps_rdf_soft_bwd(grid.handle, _ptr(dsrf), mp, float(dsrf_min), float(sigma), float(scale),
                                 Bins(r0, dr, nb), _ptr(dLdh), _ptr(gx), _ptr(gs), _stream(stream)))
    return gx, gs


def soft_r_cut(bins, sigma: float, scale: float) -> float:
    """Grid cutoff (unscaled nm) that covers every pair of the smoothed RDF."""
    r0, dr, nb = bins
    return (r0 + nb * dr + 6.0 * sigma) / scale * (1.0 + 1e-5)


def _soft_function():
    import torch

    class SoftRDF(torch.autograd.Function):
        """h = SoftRDF.apply(xyz, scale, type, dsrf, nbr_types, ctr_types, dsrf_min, sigma, bins).

        xyz: float32 CUDA [n, 3]; scale: 0-d or 1-element float tensor (its value is read on the host).
        Forward builds the cell grid for the current positions and runs ps_rdf_soft_fwd; backward
        reuses that grid and runs ps_rdf_soft_bwd (pairs recomputed).  Gradients flow to xyz and scale.
        """

        @staticmethod
        def forward(ctx, xyz, scale, type_, dsrf, nbr_types, ctr_types, dsrf_min, sigma, bins):
            s = float(scale.detach().reshape(-1)[0].item())
            xyz_c = xyz.detach().contiguous()
            g = Grid(xyz_c.shape[0]).build(xyz_c, type_, nbr_types, soft_r_cut(bins, sigma, s))
            h = soft_rdf_fwd(g, dsrf, ctr_types, dsrf_min, sigma, s, bins)
            ctx.grid, ctx.args = g, (dsrf, ctr_types, dsrf_min, sigma, s, bins)
            ctx.scale_shape, ctx.scale_dev = scale.shape, scale.device
            return h

        @staticmethod
        def backward(ctx, grad_h):
            dsrf, ctr_types, dsrf_min, sigma, s, bins = ctx.args
            gx, gs = soft_rdf_bwd(ctx.grid, dsrf, ctr_types, dsrf_min, sigma, s, bins, grad_h)
            ctx.grid = None
            return gx, gs.reshape(ctx.scale_shape).to(ctx.scale_dev), None, None, None, None, None, None, None

    return SoftRDF


_SoftRDF = None


def soft_rdf(xyz, scale, type_, dsrf, nbr_types, ctr_types, dsrf_min, sigma, bins):
    """Differentiable Gaussian-smoothed RDF (torch.autograd.Function over ps_rdf_soft_fwd/bwd)."""
    global _SoftRDF
    if _SoftRDF is None:
        _SoftRDF = _soft_function()
    return _SoftRDF.apply(xyz, scale, type_, dsrf, nbr_types, ctr_types, dsrf_min, sigma, bins)


class Batch:
    """Batched sweeps over many ROIs (ps_batch_create / ps_batch_run).

    datasets: list of (xyz, type, dsrf) CUDA tensors (dsrf may be None).
    bins: (r0, dr, n_bins) at the largest r_max; rmax_bins: ascending bin counts (last = n_bins);
    dsrf_min: ascending thresholds; pairs: list of (ctr_types, nbr_types); k_max: k = 1..k_max.
    run() returns an int64 CUDA tensor [n_roi, n_pairs, n_rmax, n_dsrf, rec] with
    rec = n_bins + k_max * n_bins + 4 + 2 * k_max (rdf | knn | meta, as ps_spatstat).
    """

    def __init__(self, datasets, bins, rmax_bins, dsrf_min, pairs, k_max, cell_scale=1.0):
        self._refs = list(datasets)
        ds = (Dataset * len(datasets))()
        for i, (X, T, D) in enumerate(datasets):
            _check_cloud(X, T, D)
            ds[i] = Dataset(X.data_ptr(), T.data_ptr(), D.data_ptr() if D is not None else None, X.shape[0])
        sw = Sweep()
        sw.struct_size = ctypes.sizeof(Sweep)
        sw.bins = Bins(*bins)
        sw.n_rmax = len(rmax_bins)
        for i, r in enumerate(rmax_bins):
            sw.rmax_bins[i] = int(r)
        sw.n_dsrf = len(dsrf_min)
        for i, d in enumerate(dsrf_min):
            sw.dsrf_min[i] = float(d)
        sw.n_pairs = len(pairs)
        for p, (c, n) in enumerate(pairs):
            mc, mn = type_mask(c), type_mask(n)
            for w in range(4):
                sw.ctr_mask[p][w] = int(mc[w])
                sw.nbr_mask[p][w] = int(mn[w])
        sw.k_max = int(k_max)
        sw.cell_scale = float(cell_scale)
        h = ctypes.c_void_p()
        _check(lib().ps_batch_create(ds, len(datasets), ctypes.byref(sw), ctypes.byref(h)))
        self._h = h
        self.shape = (len(datasets), len(pairs), len(rmax_bins), len(dsrf_min),
                      bins[2] + k_max * bins[2] + META_HEAD + 2 * k_max)
        self.bins, self.k_max = bins, k_max

    def run(self, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty(self.shape, dtype=torch.int64, device=self._refs[0][0].device)
        assert out.numel() == lib().ps_batch_out_len(self._h)
        _check(lib().ps_batch_run(self._h, _ptr(out), _stream(stream)))
        return out

    def split(self, rec):
        """rec [..., rec_len] -> (rdf [..., n_bins], knn [..., k_max, n_bins], meta [..., 4 + 2 k_max])."""
        nb, k = self.bins[2], self.k_max
        return rec[..., :nb], rec[..., nb:nb + k * nb].reshape(*rec.shape[:-1], k, nb), rec[..., nb + k * nb:]

    def close(self):
        if self._h:
            _check(lib().ps_batch_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.ps_batch_destroy(self._h)
        except Exception:
            pass


def shuffle_labels(type_, seed: int, with_perm: bool = False, stream=None):
    """Randomised labels (ps_shuffle_labels): type_out[i] = type_[perm(i)]; returns type_out (and perm)."""
    import torch

    out = torch.empty_like(type_)
    perm = torch.empty(type_.shape[0], dtype=torch.int32, device=type_.device) if with_perm else None
    _check(lib().ps_shuffle_labels(_ptr(type_), _ptr(out), type_.shape[0], int(seed) & 0xFFFFFFFFFFFFFFFF,
                                   _ptr(perm), _stream(stream)))
    return (out, perm) if with_perm else out
