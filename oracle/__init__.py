"""Oracle for the spatial-statistics hot path — TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package.  The product path (the CUDA library and its Python binding)
never imports, links or executes anything here, and this package imports
nothing from the product.

`oracle.c` is plain single-threaded C written from the paper's definitions of
the kNN and RDF statistics (Methods, "Descriptive, two-point spatial
statistics, and clustering"; Suppl. Figs. SchematicKNN/SchematicRDF), with
the d_srf edge rule (Methods, "Ion-to-edge distancing") and per-ROI
enumeration (Suppl., "Customized user defined batch processing queues").
The spatial distribution map (the 3-D two-point statistic, same Methods
passage; voxelised displacements within the ROI radius R, Results on strong
scaling) bins the float32 displacement of every in-range pair.  Maximum-separation
clustering (same Methods passage: DBScan with d_max and N_min) labels the
connected components of the d_max graph.
The smoothed-RDF functions are FP64.  The g(r) normalisation (FP64) follows a
reading, since the paper gives no formula; it is pinned by the uniform-density
limit g -> 1 of a Poisson process and by the lattice's shell counts.  Every
function is pinned by the tests under tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, u32, f32, f64 = ctypes.c_int64, ctypes.c_uint32, ctypes.c_float, ctypes.c_double
        lib.orc_edges.argtypes = [f64, f64, u32, P]
        lib.orc_edges.restype = None
        sig = [P, P, P, i64, P, P, f32, f64, f64, u32, P, u32, P, P, P, P, P, P]
        lib.orc_spatstat.argtypes = sig
        lib.orc_spatstat.restype = ctypes.c_int
        lib.orc_spatstat_brute.argtypes = sig
        lib.orc_spatstat_brute.restype = ctypes.c_int
        lib.orc_central_brute.argtypes = [P, P, i64, i64, P, f64, f64, u32, P, u32, P, P, P]
        lib.orc_central_brute.restype = ctypes.c_int
        lib.orc_soft_fwd.argtypes = [P, P, P, i64, P, P, f32, f64, f64, f64, f64, u32, P]
        lib.orc_soft_fwd.restype = ctypes.c_int
        lib.orc_soft_bwd.argtypes = [P, P, P, i64, P, P, f32, f64, f64, f64, f64, u32, P, P, P]
        lib.orc_soft_bwd.restype = ctypes.c_int
        lib.orc_sdm_edges.argtypes = [f64, u32, P]
        lib.orc_sdm_edges.restype = None
        lib.orc_sdm.argtypes = [P, P, P, i64, P, P, f32, f64, f64, u32, P, P]
        lib.orc_sdm.restype = ctypes.c_int
        lib.orc_cluster.argtypes = [P, P, P, i64, P, f64, u32, f32, u32, P, P, P, P]
        lib.orc_cluster.restype = ctypes.c_int
        lib.orc_label_perm.argtypes = [i64, ctypes.c_uint64, P]
        lib.orc_label_perm.restype = None
        lib.orc_shuffle_labels.argtypes = [P, P, i64, ctypes.c_uint64]
        lib.orc_shuffle_labels.restype = ctypes.c_int
        lib.orc_rdf_normalise.argtypes = [P, u32, f64, f64, ctypes.c_uint64, ctypes.c_uint64, f64, P]
        lib.orc_rdf_normalise.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def type_mask(types) -> np.ndarray:
    """256-bit type set as 4 x uint64; `types` is an iterable of labels or 'all'."""
    m = np.zeros(4, dtype=np.uint64)
    if isinstance(types, str) and types == "all":
        m[:] = np.uint64(0xFFFFFFFFFFFFFFFF)
        return m
    for t in types:
        t = int(t)
        m[t >> 6] |= np.uint64(1) << np.uint64(t & 63)
    return m


def edges(r0: float, dr: float, n_bins: int) -> np.ndarray:
    E = np.empty(n_bins + 1, dtype=np.float32)
    _load().orc_edges(float(r0), float(dr), int(n_bins), _ptr(E))
    return E


def _prep(xyz, type_, dsrf):
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    type_ = np.ascontiguousarray(type_, dtype=np.uint8)
    dsrf = np.ascontiguousarray(dsrf, dtype=np.float32)
    n = xyz.shape[0]
    if type_.shape[0] != n or dsrf.shape[0] != n:
        raise ValueError("xyz, type and dsrf lengths differ")
    return xyz, type_, dsrf, n


def spatstat(xyz, type_, dsrf, ctr_types, nbr_types, dsrf_min, r0, dr, n_bins, ks=(), per_central=False,
             brute=False):
    """Exact RDF and kNN histograms (see oracle.c).  Returns a dict of numpy arrays."""
    xyz, type_, dsrf, n = _prep(xyz, type_, dsrf)
    ks_a = np.ascontiguousarray(ks, dtype=np.uint32)
    nk = ks_a.shape[0]
    rdf = np.zeros(n_bins, np.uint64)
    rdf_meta = np.zeros(3, np.uint64)
    knn = np.zeros((max(nk, 1), n_bins), np.uint64)
    knn_meta = np.zeros((max(nk, 1), 2), np.uint64)
    kth = np.full((max(nk, 1), n), np.nan, np.float32) if per_central else None
    nw = np.full(n, 0xFFFFFFFF, np.uint32) if per_central else None
    fn = _load().orc_spatstat_brute if brute else _load().orc_spatstat
    rc = fn(_ptr(xyz), _ptr(type_), _ptr(dsrf), n, _ptr(type_mask(ctr_types)), _ptr(type_mask(nbr_types)),
            float(dsrf_min), float(r0), float(dr), int(n_bins), _ptr(ks_a), nk, _ptr(rdf), _ptr(rdf_meta),
            _ptr(knn), _ptr(knn_meta), _ptr(kth), _ptr(nw))
    if rc != 0:
        raise RuntimeError(f"oracle spatstat failed: {rc}")
    out = dict(rdf=rdf, n_central=int(rdf_meta[0]), n_pairs=int(rdf_meta[1]), rdf_below=int(rdf_meta[2]),
               knn=knn[:nk], not_found=knn_meta[:nk, 0].copy(), knn_below=knn_meta[:nk, 1].copy())
    if per_central:
        out["kth_d2"] = kth[:nk]
        out["n_within"] = nw
    return out


def central_brute(xyz, type_, i, nbr_types, r0, dr, n_bins, ks=(), with_rdf=False):
    """One central ion by brute force; returns (n_within, kth_d2[n_k], rdf_i or None)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    type_ = np.ascontiguousarray(type_, dtype=np.uint8)
    ks_a = np.ascontiguousarray(ks, dtype=np.uint32)
    kth = np.zeros(max(ks_a.shape[0], 1), np.float32)
    nw = np.zeros(1, np.uint32)
    rdf_i = np.zeros(n_bins, np.uint64) if with_rdf else None
    rc = _load().orc_central_brute(_ptr(xyz), _ptr(type_), xyz.shape[0], int(i), _ptr(type_mask(nbr_types)),
                                   float(r0), float(dr), int(n_bins), _ptr(ks_a), ks_a.shape[0], _ptr(kth),
                                   _ptr(nw), _ptr(rdf_i))
    if rc != 0:
        raise RuntimeError(f"oracle central_brute failed: {rc}")
    return int(nw[0]), kth[: ks_a.shape[0]], rdf_i


def soft_fwd(xyz, type_, dsrf, ctr_types, nbr_types, dsrf_min, sigma, scale, r0, dr, n_bins):
    """FP64 Gaussian-smoothed RDF h[b]."""
    xyz, type_, dsrf, n = _prep(xyz, type_, dsrf)
    h = np.zeros(n_bins, np.float64)
    rc = _load().orc_soft_fwd(_ptr(xyz), _ptr(type_), _ptr(dsrf), n, _ptr(type_mask(ctr_types)),
                              _ptr(type_mask(nbr_types)), float(dsrf_min), float(sigma), float(scale), float(r0),
                              float(dr), int(n_bins), _ptr(h))
    if rc != 0:
        raise RuntimeError(f"oracle soft_fwd failed: {rc}")
    return h


def soft_bwd(xyz, type_, dsrf, ctr_types, nbr_types, dsrf_min, sigma, scale, r0, dr, n_bins, G):
    """FP64 adjoint: returns (dL/dxyz [n,3], dL/ds) for upstream G = dL/dh."""
    xyz, type_, dsrf, n = _prep(xyz, type_, dsrf)
    G = np.ascontiguousarray(G, dtype=np.float64)
    gx = np.zeros((n, 3), np.float64)
    gs = np.zeros(1, np.float64)
    rc = _load().orc_soft_bwd(_ptr(xyz), _ptr(type_), _ptr(dsrf), n, _ptr(type_mask(ctr_types)),
                              _ptr(type_mask(nbr_types)), float(dsrf_min), float(sigma), float(scale), float(r0),
                              float(dr), int(n_bins), _ptr(G), _ptr(gx), _ptr(gs))
    if rc != 0:
        raise RuntimeError(f"oracle soft_bwd failed: {rc}")
    return gx, float(gs[0])


def sdm_edges(w: float, n_vox: int) -> np.ndarray:
    """Voxel edges V[m] = (float)((m - n_vox/2) * w), m = 0..n_vox (see oracle.c)."""
    V = np.empty(n_vox + 1, dtype=np.float32)
    _load().orc_sdm_edges(float(w), int(n_vox), _ptr(V))
    return V


def sdm(xyz, type_, dsrf, ctr_types, nbr_types, dsrf_min, r_max, w, n_vox):
    """Spatial distribution map H[n_vox, n_vox, n_vox] (indexed [mz, my, mx]) and
    meta = {n_central, pairs in the map, pairs outside the voxel cube}."""
    xyz, type_, dsrf, n = _prep(xyz, type_, dsrf)
    H = np.zeros((n_vox, n_vox, n_vox), np.uint64)
    meta = np.zeros(3, np.uint64)
    rc = _load().orc_sdm(_ptr(xyz), _ptr(type_), _ptr(dsrf), n, _ptr(type_mask(ctr_types)),
                         _ptr(type_mask(nbr_types)), float(dsrf_min), float(r_max), float(w), int(n_vox), _ptr(H),
                         _ptr(meta))
    if rc != 0:
        raise RuntimeError(f"oracle sdm failed: {rc}")
    return H, meta


def cluster(xyz, type_, dsrf, types, d_max, n_min, dsrf_min=0.0, hist_len=1024):
    """Maximum-separation clustering (see oracle.c).  Returns dict(label uint32 [n], size_hist,
    interior_hist uint64 [hist_len], n_set, n_clusters, n_clustered, n_interior)."""
    xyz, type_, dsrf, n = _prep(xyz, type_, dsrf)
    label = np.empty(n, np.uint32)
    sh = np.zeros(hist_len, np.uint64)
    ih = np.zeros(hist_len, np.uint64)
    meta = np.zeros(4, np.uint64)
    rc = _load().orc_cluster(_ptr(xyz), _ptr(type_), _ptr(dsrf), n, _ptr(type_mask(types)), float(d_max), int(n_min),
                             float(dsrf_min), int(hist_len), _ptr(label), _ptr(sh), _ptr(ih), _ptr(meta))
    if rc != 0:
        raise RuntimeError(f"oracle cluster failed: {rc}")
    return dict(label=label, size_hist=sh, interior_hist=ih, n_set=int(meta[0]), n_clusters=int(meta[1]),
                n_clustered=int(meta[2]), n_interior=int(meta[3]))


def label_perm(n: int, seed: int) -> np.ndarray:
    """The pseudo-random permutation of [0, n) used for randomised labels (see oracle.c)."""
    perm = np.empty(max(n, 1), np.uint32)
    _load().orc_label_perm(int(n), int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(perm))
    return perm[:n]


def shuffle_labels(type_, seed: int) -> np.ndarray:
    """Randomised labels out[i] = type[perm(i)]."""
    t = np.ascontiguousarray(type_, dtype=np.uint8)
    out = np.empty_like(t)
    rc = _load().orc_shuffle_labels(_ptr(t), _ptr(out), t.shape[0], int(seed) & 0xFFFFFFFFFFFFFFFF)
    if rc != 0:
        raise RuntimeError(f"oracle shuffle_labels failed: {rc}")
    return out


def rdf_normalise(rdf, r0: float, dr: float, n_central: int, n_nbr: int, volume: float) -> np.ndarray:
    """g_b = H[b] / (n_central * (n_nbr / volume) * 4/3 pi (e_{b+1}^3 - e_b^3)), FP64 (orc_rdf_normalise)."""
    h = np.ascontiguousarray(rdf, np.uint64)
    g = np.empty(h.shape[0], np.float64)
    rc = _load().orc_rdf_normalise(_ptr(h), h.shape[0], float(r0), float(dr), int(n_central), int(n_nbr),
                                   float(volume), _ptr(g))
    if rc:
        raise ValueError(f"orc_rdf_normalise failed: {rc}")
    return g
