"""Slab sharding of one specimen over ranks: the paper's spatial splitting (Methods, "Spatial
splitting": the point cloud is cut along the specimen axis into slabs that hold equal numbers
of ions, each process works on its own slab, results are combined at the end) applied across
GPUs.

Host-side partition logic only; every rank then runs the same library calls on its own data:
  * the needle is generated in z layers (one fcc cell high); the layers are cut into `world`
    consecutive slabs of (nearly) equal ion count;
  * a rank holds its core layers plus a halo of `halo_layers` layers on each side, deep enough
    that every neighbour within r_cut of a core ion is present (the halo covers r_cut plus
    15 standard deviations of the z jitter on both sides);
  * halo ions carry d_srf = NaN, which no threshold admits, so only core ions are centrals and
    every central is a central on exactly one rank;
  * the ranks' integer histograms and counters add up exactly to the whole specimen's (one
    all-reduce, sum; the device status words are combined with max).
"""
from __future__ import annotations

import math

import numpy as np


def layer_cuts(counts, parts: int, lo: int = 0, hi: int | None = None) -> list:
    """Cut layers [lo, hi) into `parts` consecutive slabs of nearly equal ion count.
    Returns parts + 1 ascending layer indices, first lo, last hi (a slab may be empty)."""
    counts = np.asarray(counts, np.int64)
    hi = counts.shape[0] if hi is None else hi
    if parts < 1 or not 0 <= lo <= hi <= counts.shape[0]:
        raise ValueError("need parts >= 1 and 0 <= lo <= hi <= layers")
    cum = np.concatenate([[0], np.cumsum(counts[lo:hi])])
    total = int(cum[-1])
    cuts = [lo]
    for r in range(1, parts):
        target = total * r / parts
        k = int(np.searchsorted(cum, target, side="left"))
        if k > 0 and (k >= cum.shape[0] or target - cum[k - 1] < cum[k] - target):
            k -= 1  # the nearer of the two layer boundaries around the target
        cuts.append(max(cuts[-1], min(hi, lo + k)))
    cuts.append(hi)
    return cuts


def halo_layers(layer_height: float, r_cut: float, sig_z: float, n_sigma: float = 15.0) -> int:
    """Layers on each side of a slab that hold every neighbour within r_cut of its core ions:
    an ion of layer k lies within n_sigma * sig_z of [k h, (k + 1) h), so a neighbour of a core
    ion can lie at most r_cut + 2 n_sigma sig_z beyond the core's last layer boundary."""
    if not (layer_height > 0 and r_cut >= 0 and sig_z >= 0):
        raise ValueError("bad halo parameters")
    return int(math.ceil((r_cut + 2.0 * n_sigma * sig_z) / layer_height)) + 1


def rank_layers(cuts, rank: int, halo: int, n_layers: int):
    """(first, end) of the generated layers and (core_first, core_end) of the core of `rank`."""
    c0, c1 = cuts[rank], cuts[rank + 1]
    return max(0, c0 - halo), min(n_layers, c1 + halo), c0, c1


def mark_halo(counts, k0: int, c0: int, c1: int, dsrf: np.ndarray) -> tuple:
    """Set d_srf = NaN for the ions of the halo layers of a slab generated from layer k0 on, so
    that only the core layers [c0, c1) hold centrals.  Returns the core's index range in the
    slab's arrays."""
    counts = np.asarray(counts, np.int64)
    i0 = int(counts[k0:c0].sum())
    i1 = i0 + int(counts[c0:c1].sum())
    dsrf[:i0] = np.float32(np.nan)
    dsrf[i1:] = np.float32(np.nan)
    return i0, i1


def slab_needle(p, counts, cuts, rank: int, halo: int, alloc=None):
    """Generate the slab of `rank` (core + halo layers) of the needle with parameters p.

    alloc(n) -> (xyz [n, 3] float32, type [n] uint8, dsrf [n] float32) writable numpy arrays
    (e.g. views of pinned host memory); default: new numpy arrays.  Returns (xyz, type, dsrf,
    (i0, i1)) with the halo's d_srf set to NaN and (i0, i1) the core's index range."""
    from . import specimen

    n_layers = len(counts)
    k0, k1, c0, c1 = rank_layers(cuts, rank, halo, n_layers)
    n = int(np.asarray(counts[k0:k1], np.int64).sum())
    if alloc is None:
        xyz, t, d = np.empty((n, 3), np.float32), np.empty(n, np.uint8), np.empty(n, np.float32)
    else:
        xyz, t, d = alloc(n)
    if n:
        specimen.needle_fill(p, k0, k1, np.asarray(counts, np.int64), xyz.ctypes.data, t.ctypes.data, d.ctypes.data)
    core = mark_halo(counts, k0, c0, c1, d)
    return xyz, t, d, core


SUM_KEYS = ("rdf", "knn")


def combine(dist, out: dict, device=None) -> None:
    """Add the ranks' results in place: histograms and meta counters summed, the meta status
    word (index 3) combined with max.  out holds int64 tensors rdf, knn (may be None), meta."""
    if dist is None:
        return
    import torch

    parts = [out[k].reshape(-1) for k in SUM_KEYS if out.get(k) is not None]
    meta = out["meta"]
    status = meta[3:4].clone()
    flat = torch.cat(parts + [meta.reshape(-1)])
    flat[-meta.numel() + 3] = 0
    host = dist.get_backend() == "gloo" and flat.is_cuda  # gloo sums host tensors
    if host:
        flat, status = flat.cpu(), status.cpu()
    dist.all_reduce(flat)
    dist.all_reduce(status, op=dist.ReduceOp.MAX)
    if host:
        flat, status = flat.to(meta.device), status.to(meta.device)
    o = 0
    for k in SUM_KEYS:
        if out.get(k) is not None:
            n = out[k].numel()
            out[k].copy_(flat[o:o + n].view_as(out[k]))
            o += n
    meta.copy_(flat[o:o + meta.numel()])
    meta[3:4].copy_(status)
