"""Build libps.so (the CUDA library) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libps.so")
ROOT = os.path.dirname(PKG)

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code: no contraction either (the edge tables are computed on the host and on the device alike)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


# Translation units whose float32 arithmetic must not be contracted into FMA:
# the exact path compares squared distances bit for bit, and ptxas fuses packed
# (f32x2) multiplies and adds even when they carry an explicit rounding modifier.
NO_FMA = {"ps_query.cu", "ps_grid.cu", "ps_batch.cu", "ps_sdm.cu", "ps_cluster.cu", "ps_peaks.cu", "ps_finalise.cu"}


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every csrc/*.cu in parallel, then link libps.so.  Returns its path.

    Concurrent callers (one per rank) serialise on a lock file."""
    import fcntl

    if not force and not _stale(LIB):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with open(os.path.join(BUILD, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            if force or _stale(LIB):
                _build_locked(verbose, extra_flags)
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)
    return LIB


def _build_locked(verbose, extra_flags):
    srcs = _sources()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        fmad = ["-fmad=false", "-Xptxas", "--fmad=false"] if os.path.basename(src) in NO_FMA else []
        cmd = [NVCC, *ARCH, *FLAGS, *fmad, *extra_flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
