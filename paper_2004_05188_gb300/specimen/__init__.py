"""Seeded synthetic specimens: the input clouds of every workload.

This module generates inputs only (float32 xyz in nm, uint8 type, float32
d_srf); it holds none of the spatial-statistics arithmetic.  Both the CUDA
path and the oracle consume what it produces.  Generation runs in C
(`specimen.c`, counter-based randomness, OpenMP), so a cloud is identical for
every thread count.

Type labels: 0 = Al, 1 = Sc, 2 = Si.

Workloads (sizes of the paper's synthetic quartet, Methods "Benchmarking all
functionality with synthetic datasets"; the shapes and rates below are the
configurations this library is measured on):
  * cylinder_small(): 200,000 ions, homogeneous Poisson in a cylinder
    R = 10 nm, H = 15.9 nm (40 ions/nm^3), Al 97 % / Sc 2 % / Si 1 %.
  * needle(...): conical frustum (tip radius, half-angle, height), fcc Al
    lattice a = 0.404 nm thinned to 30 ions/nm^3, Gaussian jitter
    (0.3 nm in x, y; 0.1 nm in z), Al3Sc precipitates (Poisson centres at
    1e-3 /nm^3, log-normal radius median 2 nm, sigma 0.3, 25 % Sc inside),
    matrix Sc 0.3 %, Si 0.2 %.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "specimen.c")
_LIB = os.path.join(_HERE, "libpsgen.so")

AL, SC, SI = 0, 1, 2
FCC_A = 0.404
FCC_DENSITY = 4.0 / FCC_A**3  # sites per nm^3


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class NeedleParams(ctypes.Structure):
    _fields_ = [("r_top", ctypes.c_double), ("half_angle", ctypes.c_double), ("height", ctypes.c_double),
                ("a", ctypes.c_double), ("keep", ctypes.c_double), ("sig_xy", ctypes.c_double),
                ("sig_z", ctypes.c_double), ("prec_density", ctypes.c_double), ("prec_median", ctypes.c_double),
                ("prec_sigma", ctypes.c_double), ("in_sc", ctypes.c_double), ("out_sc", ctypes.c_double),
                ("out_si", ctypes.c_double), ("seed", ctypes.c_uint64)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, i64, f64, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
        lib.psg_cylinder.argtypes = [u64, i64, f64, f64, P, ctypes.c_int, P, P, P]
        lib.psg_cube.argtypes = [u64, i64, f64, P, ctypes.c_int, P, P, P]
        lib.psg_needle_layers.argtypes = [ctypes.POINTER(NeedleParams)]
        lib.psg_needle_layers.restype = i64
        lib.psg_needle_plan.argtypes = [ctypes.POINTER(NeedleParams), P]
        lib.psg_needle_plan.restype = i64
        lib.psg_needle_fill.argtypes = [ctypes.POINTER(NeedleParams), i64, i64, P, P, P, P]
        lib.psg_needle_precipitates.argtypes = [ctypes.POINTER(NeedleParams)]
        lib.psg_needle_precipitates.restype = i64
        lib.psg_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(_load().psg_threads())


def cylinder(seed: int, n: int, R: float, H: float, type_prob=(0.97, 0.02, 0.01)):
    """Homogeneous Poisson cylinder; d_srf = min(R - rho, z, H - z)."""
    xyz = np.empty((n, 3), np.float32)
    t = np.empty(n, np.uint8)
    d = np.empty(n, np.float32)
    pr = np.ascontiguousarray(type_prob, np.float64)
    rc = _load().psg_cylinder(seed, n, R, H, _p(pr), pr.shape[0], _p(xyz), _p(t), _p(d))
    if rc:
        raise RuntimeError(f"psg_cylinder failed: {rc}")
    return xyz, t, d


def cube(seed: int, n: int, L: float, type_prob=(1.0,)):
    """Homogeneous Poisson cube [0, L)^3; d_srf = distance to the nearest face."""
    xyz = np.empty((n, 3), np.float32)
    t = np.empty(n, np.uint8)
    d = np.empty(n, np.float32)
    pr = np.ascontiguousarray(type_prob, np.float64)
    rc = _load().psg_cube(seed, n, L, _p(pr), pr.shape[0], _p(xyz), _p(t), _p(d))
    if rc:
        raise RuntimeError(f"psg_cube failed: {rc}")
    return xyz, t, d


def simple_cubic(m: int, a: float = 0.25, offset: float = 0.125, type_label: int = 0):
    """m^3 simple-cubic lattice (i, j, k) * a + offset; d_srf = distance to the block faces."""
    g = np.arange(m, dtype=np.float64) * a + offset
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float32)
    L = m * a
    d = np.minimum(xyz, L - xyz).min(axis=1).astype(np.float32)
    return xyz, np.full(xyz.shape[0], type_label, np.uint8), d


def needle_params(r_top=20.0, half_angle_deg=10.0, height=100.0, seed=2, density=30.0, prec_density=1e-3,
                  prec_median=2.0, prec_sigma=0.3, in_sc=0.25, out_sc=0.003, out_si=0.002, sig_xy=0.3,
                  sig_z=0.1) -> NeedleParams:
    return NeedleParams(r_top, math.radians(half_angle_deg), height, FCC_A, density / FCC_DENSITY, sig_xy, sig_z,
                        prec_density, prec_median, prec_sigma, in_sc, out_sc, out_si, seed)


def frustum_volume(r_top: float, half_angle_deg: float, height: float) -> float:
    rb = r_top + height * math.tan(math.radians(half_angle_deg))
    return math.pi * height / 3.0 * (rb * rb + rb * r_top + r_top * r_top)


def height_for(n_ions: float, r_top: float, half_angle_deg: float, density: float = 30.0) -> float:
    """Frustum height whose expected ion count at `density` is n_ions (bisection)."""
    lo, hi = 0.0, 1.0
    while frustum_volume(r_top, half_angle_deg, hi) * density < n_ions:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if frustum_volume(r_top, half_angle_deg, mid) * density < n_ions:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def needle_plan(p: NeedleParams) -> np.ndarray:
    nk = _load().psg_needle_layers(ctypes.byref(p))
    if nk < 0:
        raise RuntimeError("bad needle parameters")
    counts = np.zeros(nk, np.int64)
    tot = _load().psg_needle_plan(ctypes.byref(p), _p(counts))
    if tot < 0:
        raise RuntimeError("psg_needle_plan failed")
    return counts


def needle_fill(p: NeedleParams, k0: int, k1: int, counts: np.ndarray, xyz_addr: int, type_addr: int,
                dsrf_addr: int) -> None:
    """Write the ions of lattice layers [k0, k1) to raw host addresses (contiguous, starting at 0)."""
    rc = _load().psg_needle_fill(ctypes.byref(p), k0, k1, _p(counts), ctypes.c_void_p(xyz_addr),
                                 ctypes.c_void_p(type_addr), ctypes.c_void_p(dsrf_addr))
    if rc:
        raise RuntimeError(f"psg_needle_fill failed: {rc}")


def needle(p: NeedleParams):
    counts = needle_plan(p)
    n = int(counts.sum())
    xyz = np.empty((n, 3), np.float32)
    t = np.empty(n, np.uint8)
    d = np.empty(n, np.float32)
    needle_fill(p, 0, counts.shape[0], counts, xyz.ctypes.data, t.ctypes.data, d.ctypes.data)
    return xyz, t, d


def needle_precipitates(p: NeedleParams) -> int:
    return int(_load().psg_needle_precipitates(ctypes.byref(p)))


# ---------------------------------------------------------------------------
# The measured workloads
# ---------------------------------------------------------------------------

def cylinder_small(seed: int = 1):
    """200,000-ion Poisson cylinder, R = 10 nm, H = 15.9 nm, Al/Sc/Si = 97/2/1 %."""
    return cylinder(seed, 200_000, 10.0, 15.9, (0.97, 0.02, 0.01))


def needle_8m_params(seed: int = 2) -> NeedleParams:
    """Needle: tip radius 20 nm, half-angle 10 deg, height 100 nm (~8.07e6 ions)."""
    return needle_params(20.0, 10.0, 100.0, seed)


def needle_10m_params(seed: int = 4) -> NeedleParams:
    """The same needle with its height scaled to 1e7 expected ions."""
    return needle_params(20.0, 10.0, height_for(1e7, 20.0, 10.0), seed)


def needle_2g_params(seed: int = 5) -> NeedleParams:
    """Full-scale needle: tip radius 40 nm, half-angle 15 deg, height for 2e9 ions."""
    return needle_params(40.0, 15.0, height_for(2e9, 40.0, 15.0), seed)


def roi_sizes(n_rois: int = 256, lo: float = 1e4, hi: float = 1e7, seed0: int = 1000):
    """Log-uniform ROI sizes, one seeded draw per ROI (seed0 + i)."""
    out = []
    for i in range(n_rois):
        u = np.random.default_rng(seed0 + i).random()
        out.append(int(round(lo * (hi / lo) ** u)))
    return out


def roi(i: int, n: int, seed0: int = 1000):
    """ROI i of the batched workload: even i a needle scaled isotropically from
    the 8e6-ion needle to n expected ions, odd i a Poisson cylinder with the
    small cylinder's aspect ratio, density and composition at n ions."""
    seed = seed0 + i
    if i % 2 == 0:
        f = (n / (30.0 * frustum_volume(20.0, 10.0, 100.0))) ** (1.0 / 3.0)
        return needle(needle_params(20.0 * f, 10.0, 100.0 * f, seed))
    R = (n / (40.0 * math.pi * 1.59)) ** (1.0 / 3.0)
    return cylinder(seed, n, R, 1.59 * R, (0.97, 0.02, 0.01))
