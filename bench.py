#!/usr/bin/env python
"""Benchmark of the exact kNN + RDF spatial-statistics path on GB300.

Default workload: the full-scale needle of 2e9 ions (tip radius 40 nm,
half-angle 15 deg, height 812.6 nm, 30 ions/nm^3, Al3Sc precipitates), type
combinations all-all and Sc-Sc, k = 10, RDF on r = [0, 0.01, 2] nm, central
ions with d_srf >= 2 nm.  One step = for each combination: build the
neighbour cell grid (binner) and run the kNN + RDF query (central list +
query kernel), i.e. every step of the exact path, with inputs resident in
HBM.  With N ranks the specimen is cut into N z-slabs of equal ion count
(each rank generates and holds only its slab plus an r_cut halo) and the
integer results are summed with one all-reduce per combination: strong
scaling of one specimen.

value   = ion queries (central ions evaluated, summed over the combinations)
          per second of device time, max over ranks.
e2e     = the same metric through the public Python API with the inputs in
          pinned host memory: H2D copy + both combinations + D2H of results.
roofline: the query kernel (the dominant family), timed with CUDA events
          around every launch on its stream inside the timed region, against
          the FP32 add/multiply throughput measured on the GPU at hand; beside
          it the shared-atomic bound of its RDF increments and the HBM
          fraction of the build kernels.
cpu_baseline: the oracle (C) on a bounded z-slab sample of the same needle,
          on every host core (one share of the sample's centrals per thread,
          exact sum).
secondary: the 8.07e6-ion needle (Sc-Sc + Si-Si, k = 1, 5, 10) and the
          2e5-ion cylinder (all-all), each step replayed from a CUDA graph.
forms:  the smoothed RDF (1e7 needle), the batched sweep (256 ROIs), the
          spatial distribution map and the clustering sweep (8e6 needle).

--impl reference runs the oracle as the comparison arm on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2

WORKLOADS = {
    "needle2g": dict(
        desc="needle 2e9 ions (r_tip 40 nm, 15 deg, h 812.6 nm, 30/nm^3, Al3Sc precipitates); all-all + Sc-Sc; "
             "kNN k=10 + RDF r=[0,0.01,2] nm; d_srf>=2 nm",
        combos=[("all-all", "all", "all"), ("Sc-Sc", [1], [1])], ks=[10], spec=(0.0, 0.01, 2.0), dsrf_min=2.0,
        sharded=True),
    "needle200m": dict(
        desc="needle 2e8 ions (r_tip 40 nm, 15 deg, height for 2e8 ions, 30/nm^3, Al3Sc precipitates); all-all + Sc-Sc; "
             "kNN k=10 + RDF r=[0,0.01,2] nm; d_srf>=2 nm",
        combos=[("all-all", "all", "all"), ("Sc-Sc", [1], [1])], ks=[10], spec=(0.0, 0.01, 2.0), dsrf_min=2.0,
        sharded=True),
    "needle8m": dict(
        desc="needle 8.07e6 ions (r_tip 20 nm, 10 deg, h 100 nm, 30/nm^3, Al3Sc precipitates); Sc-Sc + Si-Si; "
             "kNN k=1,5,10 + RDF r=[0,0.01,2] nm; d_srf>=2 nm",
        combos=[("Sc-Sc", [1], [1]), ("Si-Si", [2], [2])], ks=[1, 5, 10], spec=(0.0, 0.01, 2.0), dsrf_min=2.0),
    "needle8m-allall": dict(
        desc="needle 8.07e6 ions (r_tip 20 nm, 10 deg, h 100 nm, 30/nm^3, Al3Sc precipitates); all-all; "
             "kNN k=10 + RDF r=[0,0.01,2] nm; d_srf>=2 nm",
        combos=[("all-all", "all", "all")], ks=[10], spec=(0.0, 0.01, 2.0), dsrf_min=2.0),
    "cylinder200k": dict(
        desc="Poisson cylinder 2e5 ions (R 10 nm, H 15.9 nm, 40/nm^3); all-all; kNN k=1 + RDF r=[0,0.01,2] nm; "
             "d_srf>=1 nm",
        combos=[("all-all", "all", "all")], ks=[1], spec=(0.0, 0.01, 2.0), dsrf_min=1.0),
}
SECONDARY = ("needle8m", "cylinder200k")


def make_cloud(name: str, seed_offset: int = 0):
    from paper_2004_05188_gb300 import specimen

    if name in ("needle8m", "needle8m-allall"):
        return specimen.needle(specimen.needle_8m_params(seed=2 + seed_offset))
    if name == "cylinder200k":
        return specimen.cylinder_small(seed=1 + seed_offset)
    raise ValueError(name)


def needle_params(name: str):
    from paper_2004_05188_gb300 import specimen

    if name == "needle2g":
        return specimen.needle_2g_params()
    if name == "needle200m":
        return specimen.needle_params(40.0, 15.0, specimen.height_for(2e8, 40.0, 15.0), seed=6)
    raise ValueError(name)


def load_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json, STREAM-style copy)"
    return 6800.0, "fallback"


# the pair test d2 = ((dx*dx) + (dy*dy)) + (dz*dz): 3 sub, 3 mul, 2 add, and 1 compare against the range
FLOPS_PER_CANDIDATE = 9


def query_sources_sha256() -> str:
    """Digest of the query kernels' sources (code lines only: // comments and blank lines are
    left out, so that a comment edit keeps a record): a stored ncu traffic figure holds only for
    this code."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in ("ps_query.cu", "ps_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2004_05188_gb300", "csrc", f), encoding="utf-8") as fh:
            for line in fh:
                code = re.sub(r"//.*$", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "query_traffic.json")


def stored_traffic(workload: str, kernel_config: dict):
    """DRAM bytes per launch of the query kernels from the stored ncu record
    (profiles/query_traffic.json): {"combination": name, "kernels": {family: bytes}}, or None when
    no record was taken on these kernel sources, this workload and this kernel configuration."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        recs = json.load(f).get("records", [])
    for rec in recs:
        if (rec.get("workload") == workload and rec.get("source_sha256") == query_sources_sha256()
                and rec.get("kernel_config") == kernel_config):
            return {"combination": rec["combination"],
                    "kernels": {k: float(v["dram_bytes_read"] + v["dram_bytes_write"])
                                for k, v in rec["kernels"].items()}}
    return None


def row_widths(stencil: int, cell_scale: float):
    """Half-width of each stencil row (dy, dz) of the exact query, [dz + s][dy + s] (-1: none): the
    cells whose gap to the central cell exceeds r_cut on the cell-edge bound r_cut * cell_scale *
    (1 + 2^-10) are skipped (the library's rule, restated for the test counts)."""
    s = int(stencil)
    f = float(np.float32(cell_scale)) * (1.0 + 1.0 / 1024.0)
    lim = (1.0 + 1.0 / 1048576.0) ** 2

    def m2(d):
        m = abs(d) - 1
        return float(m * m) if m > 0 else 0.0

    out = []
    for dz in range(-s, s + 1):
        row = []
        for dy in range(-s, s + 1):
            w = -1
            for dx in range(s + 1):
                if (m2(dx) + m2(dy) + m2(dz)) * f * f < lim:
                    w = dx
            row.append(w)
        out.append(row)
    return out


def candidate_tests(X, T, D, ctr, nbr, dsrf_min, info, stencil, chunk=1 << 26, all_records=False, cell_scale=None):
    """Central x candidate tests one query makes on this grid: for every central, the neighbour
    records in the (2*stencil+1)^3 cells around its cell (clipped at the grid's faces), less the
    cells the query skips (row_widths; cell_scale None: every cell of the stencil).
    Counted with plain torch ops from the grid geometry (reporting only, untimed), in chunks of
    ions so that the temporaries stay small beside a 2e9-ion cloud.  all_records: every neighbour
    record counts as a central (no type or d_srf filter)."""
    import torch

    import paper_2004_05188_gb300 as ps

    def lut(types):
        m = ps.type_mask(types)
        return torch.tensor([bool((int(m[t >> 6]) >> (t & 63)) & 1) for t in range(256)], device=T.device)

    dims = info["dims"]
    org = torch.tensor(info["origin"], dtype=torch.float32, device=X.device)
    inv_h = float(np.float32(1.0 / float(info["cell"])))
    ln, lc = lut(nbr), lut(ctr)

    def cells(P):
        u = torch.floor((P - org) * inv_h).to(torch.int64)
        for a in range(3):
            u[:, a].clamp_(0, dims[a] - 1)
        return (u[:, 2] * dims[1] + u[:, 1]) * dims[0] + u[:, 0]

    n = X.shape[0]
    cnt = torch.zeros(info["n_cells"], dtype=torch.int64, device=X.device)
    for a in range(0, n, chunk):
        sel = ln[T[a:a + chunk].long()]
        cnt += torch.bincount(cells(X[a:a + chunk][sel]), minlength=info["n_cells"])
    cnt = cnt.view(dims[2], dims[1], dims[0])
    s = int(stencil)
    widths = row_widths(s, cell_scale) if cell_scale is not None else [[s] * (2 * s + 1)] * (2 * s + 1)
    if all(w == s for row in widths for w in row):
        for ax in range(3):  # box sum of width 2s+1 along each axis (exact, int64)
            c = torch.cumsum(torch.nn.functional.pad(cnt.movedim(ax, -1), (s + 1, s)), dim=-1)
            cnt = (c[..., 2 * s + 1:] - c[..., : -(2 * s + 1)]).movedim(-1, ax).contiguous()
            del c
    else:  # rows of their own widths: x-box sums, shifted over (dy, dz)
        acc = torch.zeros_like(cnt)
        Z, Y = dims[2], dims[1]
        for w in sorted({w for row in widths for w in row if w >= 0}):
            c = torch.cumsum(torch.nn.functional.pad(cnt, (w + 1, w)), dim=-1)
            box = torch.nn.functional.pad(c[..., 2 * w + 1:] - c[..., : -(2 * w + 1)], (0, 0, s, s, s, s))
            del c
            for dz in range(-s, s + 1):
                for dy in range(-s, s + 1):
                    if widths[dz + s][dy + s] == w:
                        acc += box[s + dz: s + dz + Z, s + dy: s + dy + Y]
            del box
        cnt = acc
    cnt = cnt.reshape(-1)
    tot = 0
    for a in range(0, n, chunk):
        if all_records:  # every neighbour record as a central (the symmetric RDF pass)
            cm = ln[T[a:a + chunk].long()]
        else:
            cm = lc[T[a:a + chunk].long()] & (D[a:a + chunk] >= dsrf_min)
        tot += int(cnt[cells(X[a:a + chunk][cm])].sum().item())
    return tot


def octant_tests(X, T, D, ctr, nbr, dsrf_min, info, chunk=1 << 26):
    """Central x candidate tests of the near kNN pass on the 2 x 2 x 2 block of cells around the
    central's nearest vertex: its cell and its neighbours on the side of its half along each axis
    (the fraction of its float32 cell coordinate (x - origin) * inv_h at or above 1/2: the upper
    neighbour), clipped at the grid's faces.  Counted like candidate_tests (reporting only; the
    kernel's vertex cells use their own float32 origin, which can move a central lying within a
    rounding error of a cell's midplane to the other block)."""
    import torch

    import paper_2004_05188_gb300 as ps

    def lut(types):
        m = ps.type_mask(types)
        return torch.tensor([bool((int(m[t >> 6]) >> (t & 63)) & 1) for t in range(256)], device=T.device)

    dims = info["dims"]
    org = torch.tensor(info["origin"], dtype=torch.float32, device=X.device)
    inv_h = torch.tensor(float(np.float32(1.0 / float(info["cell"]))), dtype=torch.float32, device=X.device)
    ln, lc = lut(nbr), lut(ctr)
    lim = torch.tensor(dims, dtype=torch.int64, device=X.device) - 1

    def coords(P):
        u = (P - org) * inv_h
        c = torch.minimum(torch.floor(u).to(torch.int64).clamp_(min=0), lim)
        return c, (u - c.to(torch.float32)) >= 0.5

    n = X.shape[0]
    cnt = torch.zeros(info["n_cells"], dtype=torch.int64, device=X.device)
    for a in range(0, n, chunk):
        sel = ln[T[a:a + chunk].long()]
        c, _ = coords(X[a:a + chunk][sel])
        cnt += torch.bincount((c[:, 2] * dims[1] + c[:, 1]) * dims[0] + c[:, 0], minlength=info["n_cells"])
    cnt = cnt.view(dims[2], dims[1], dims[0])
    tot = 0
    for octant in range(8):
        up = [(octant >> ax) & 1 for ax in range(3)]  # axis 0 = x (last tensor dim)
        box = cnt
        for ax in range(3):
            dim = 2 - ax
            pad = [0, 0] * (2 - dim) + ([0, 1] if up[ax] else [1, 0])
            padded = torch.nn.functional.pad(box, pad)
            sl = [slice(None)] * 3
            sl[dim] = slice(1, None) if up[ax] else slice(0, -1)
            box = box + padded[tuple(sl)]
        box = box.reshape(-1)
        for a in range(0, n, chunk):
            cm = lc[T[a:a + chunk].long()] & (D[a:a + chunk] >= dsrf_min)
            c, hi = coords(X[a:a + chunk][cm])
            mine = (hi[:, 0] == bool(up[0])) & (hi[:, 1] == bool(up[1])) & (hi[:, 2] == bool(up[2]))
            c = c[mine]
            tot += int(box[(c[:, 2] * dims[1] + c[:, 1]) * dims[0] + c[:, 0]].sum().item())
        del box
    return tot


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, path: str | None = None):
        import tempfile

        self.index = index
        self.proc = None
        # the raw samples are kept (a record beside the number); default: a temporary file
        self.path = path or os.path.join(tempfile.gettempdir(), f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for ln in f:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax = float(parts[1])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle arm (cpu baseline and --impl reference)
# ---------------------------------------------------------------------------
def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_run(orc, cloud, wl):
    """One oracle step over a cloud (every combination); returns the centrals evaluated."""
    xyz, t, d = cloud
    r0, dr, nb = wl["bins"]
    n = 0
    for _, ctr, nbr in wl["combos"]:
        r = orc.spatstat(xyz, t, d, ctr, nbr, wl["dsrf_min"], r0, dr, nb, wl["ks"])
        n += r["n_central"]
    return n


def needle_sample(wl_name, wl, core_layers: int, shares: int):
    """Bounded sample of the large needle for the oracle: `core_layers` lattice layers about the
    middle of its height whose ions are the centrals, with the r_cut halo of neighbour layers on
    each side, generated directly (the same ions as the full cloud's).  The centrals are split
    into `shares` strips along x of equal count (one host thread each); a strip's cloud is every
    ion of the slab within r_cut of the strip in x, so the strips add up exactly."""
    from paper_2004_05188_gb300 import shard, specimen

    p = needle_params(wl_name)
    counts = specimen.needle_plan(p)
    mid = len(counts) // 2
    lo = mid - core_layers // 2
    hi = lo + core_layers
    r0, dr, nb = wl["bins"]
    r_cut = r0 + dr * nb
    halo = shard.halo_layers(p.a, r_cut, p.sig_z)
    xyz, t, d, (i0, i1) = shard.slab_needle(p, counts, [lo, hi], 0, halo)
    x = xyz[:, 0]
    cx = np.sort(x[i0:i1])
    cuts = [-np.inf] + [float(cx[len(cx) * j // shares]) for j in range(1, shares)] + [np.inf]
    core = np.zeros(x.shape[0], bool)
    core[i0:i1] = True
    parts = []
    for j in range(shares):
        keep = (x >= cuts[j] - r_cut) & (x < cuts[j + 1] + r_cut)
        own = core[keep] & (x[keep] >= cuts[j]) & (x[keep] < cuts[j + 1])
        parts.append((xyz[keep], t[keep], np.where(own, d[keep], np.float32(np.nan)).astype(np.float32)))
    desc = (f"{core_layers} lattice layers of centrals at mid-height ({i1 - i0} ions) + {halo}-layer halo each side "
            f"({xyz.shape[0]} ions generated), centrals in {shares} strips along x with an r_cut halo each "
            f"(one host thread each)")
    return parts, desc


def small_sample(wl, cloud, frac: float, shares: int):
    """Bounded z-slab sample of a small cloud: the ions of a z-slab holding `frac` of the height are
    the centrals' candidates, with an r_cut halo; their centrals split into `shares` index ranges."""
    xyz, t, d = cloud
    z = xyz[:, 2]
    zlo, zhi = float(z.min()), float(z.max())
    z0 = zlo + 0.5 * (zhi - zlo) * (1.0 - frac)
    z1 = z0 + frac * (zhi - zlo)
    r0, dr, nb = wl["bins"]
    halo = r0 + dr * nb
    keep = (z >= z0 - halo) & (z < z1 + halo)
    core = ((z >= z0) & (z < z1))[keep]
    xs, ts, ds = xyz[keep], t[keep], np.where(core, d[keep], np.float32(np.nan)).astype(np.float32)
    idx = np.nonzero(core)[0]
    parts = []
    for j in range(shares):
        sel = idx[len(idx) * j // shares: len(idx) * (j + 1) // shares]
        dj = np.full_like(ds, np.float32(np.nan))
        dj[sel] = ds[sel]
        parts.append((xs, ts, dj))
    return parts, f"z-slab with {frac:.3f} of the height (+{halo} nm halo), centrals in {shares} shares"


def oracle_sampled(wl_name, wl, cores: int, target_s: float, cloud=None):
    """A sample sized so that one oracle step on `cores` threads takes about target_s."""
    import concurrent.futures as cf

    import oracle as orc

    orc.build()
    pool = cf.ThreadPoolExecutor(max_workers=cores)
    size = 1 if wl.get("sharded") else 0.02
    while True:
        if wl.get("sharded"):
            parts, desc = needle_sample(wl_name, wl, int(size), cores)
        else:
            parts, desc = small_sample(wl, cloud, float(size), cores)
        t0 = time.perf_counter()
        nq = sum(pool.map(lambda c: oracle_run(orc, c, wl), parts))
        dt = time.perf_counter() - t0
        full = size >= 1.0 if not wl.get("sharded") else False
        if dt >= 0.3 * target_s or full:
            break
        grow = max(2.0, 0.6 * target_s / max(dt, 1e-3))
        size = min(1.0, size * grow) if not wl.get("sharded") else max(size + 1, int(size * grow))
    return orc, parts, pool, nq, desc


def oracle_steps(orc, parts, pool, wl, n):
    """n oracle steps over the sample (one thread per share); returns (centrals per step, seconds)."""
    t0 = time.perf_counter()
    nq = 0
    for _ in range(n):
        nq = sum(pool.map(lambda c: oracle_run(orc, c, wl), parts))
    return nq, time.perf_counter() - t0


def run_reference(args, wl_name, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = host_cores()
    cloud = None if wl.get("sharded") else make_cloud(wl_name)
    orc, parts, pool, nq, desc = oracle_sampled(wl_name, wl, cores, target_s=2.0, cloud=cloud)
    oracle_steps(orc, parts, pool, wl, args.warmup)
    nq, T = oracle_steps(orc, parts, pool, wl, args.steps)
    pool.shutdown()
    v = nq * args.steps / T
    line = {
        "impl": "reference", "metric": "ion-queries/s (exact kNN+RDF)", "value": v, "unit": "ion-queries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "strong" if wl.get("sharded") else "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "sample": desc},
        "cpu_baseline": {"value": v, "unit": "ion-queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{desc}; {nq} centrals per step"},
        "e2e": {"value": v, "unit": "ion-queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def algorithmic_bytes(kid: str, st: dict, c: dict) -> float:
    """Bytes one combination's kernels of a family must move per step (reads + writes of their role).
    n: ions of the cloud, nn: neighbour-set ions, nc: centrals, cells: cells of the grid."""
    N = st["n_ions"]
    nn, nc, cells, ntm = c["n_nbr"], c["n_central"], c["n_cells"], c["n_ctr_typed"]
    if kid == "select":  # type labels of every ion; xyz of the selected; their indices written
        return N * 1 + nn * 12 + nn * 4
    if kid == "geometry":  # cell counts zeroed
        return cells * 4
    if kid == "count":  # index read, xyz gathered, count increment, (cell, rank) written
        return nn * (4 + 12 + 4 + 8)
    if kid == "scan":  # counts read, starts written; central-list cell starts from the record prefix
        return cells * (4 + 4) + cells * (4 + 4 + 4)
    if kid == "scatter":  # index, (cell, rank), start read; xyz gathered; float4 record written
        return nn * (4 + 8 + 4 + 12 + 16)
    if kid == "central":
        if c.get("subset", True):  # records read, type and d_srf gathered, prefix and central records written
            return nn * (16 + 1 + 4 + 4) + nc * 16
        return N * 1 + ntm * 4 + nc * (12 + 4 + 8) + nc * (4 + 8 + 4 + 12 + 16)
    if kid == "query":  # every record and central read once; cell starts
        return nn * 16 + nc * 16 + 2 * cells * 4
    return 0.0


def measure_soft(args, dev):
    """The differentiable form on the 1e7-ion needle: forward, loss, adjoint, against the plain exact RDF.

    All types central and neighbour, d_srf >= 2.3 nm (= stop + 6 sigma: full ROIs), sigma = 0.05 nm,
    r = [0, 0.02, 2] nm; the target g* comes from a copy of the cloud with every coordinate
    perturbed by N(0, 0.02 nm) (seed 1)."""
    import torch

    import paper_2004_05188_gb300 as ps
    from paper_2004_05188_gb300 import specimen

    p = specimen.needle_10m_params()
    xyz, t, d = specimen.needle(p)
    N = xyz.shape[0]
    bins, sigma, dmin = (0.0, 0.02, 100), 0.05, 2.3
    X = torch.from_numpy(xyz).to(dev)
    T = torch.from_numpy(t).to(dev)
    D = torch.from_numpy(d).to(dev)
    pert = (xyz + np.random.default_rng(1).normal(0.0, 0.02, xyz.shape)).astype(np.float32)
    Xp = torch.from_numpy(pert).to(dev)
    rc = ps.soft_r_cut(bins, sigma, 1.0)
    # the smoothed form's cell size (--soft-cell-scale); the plain exact RDF on half-size cells in passes
    # (its fastest form)
    g = ps.Grid(N, args.soft_cell_scale)
    gp = ps.Grid(N, args.soft_cell_scale)
    gplain = ps.Grid(N, 0.5, 0, True)
    # normalisation at fixed density (the library's g(r) finalisation, ps_rdf_normalise):
    # g_b = h_b * factor_b, factor_b = 1 / (N_c (N / V) 4/3 pi (e_{b+1}^3 - e_b^3))
    vol = specimen.frustum_volume(p.r_top, math.degrees(p.half_angle), p.height)
    gp.build(Xp, T, "all", rc)
    h_star = ps.soft_rdf_fwd(gp, D, "all", dmin, sigma, 1.0, bins)
    meta0 = ps.spatstat(g.build(X, T, "all", rc), D, "all", dmin, bins, [], rdf=True)["meta"]
    n_c = float(meta0[0].item())
    factor = ps.rdf_normalise(g, meta0, bins, vol)[1].float()
    g_star = h_star * factor
    plain_out = dict(rdf=torch.empty(bins[2], dtype=torch.int64, device=dev),
                     meta=torch.empty(ps.META_HEAD, dtype=torch.int64, device=dev))

    def fwd():
        g.build(X, T, "all", rc)
        return ps.soft_rdf_fwd(g, D, "all", dmin, sigma, 1.0, bins)

    def loss_grad(h):
        return 2.0 * (h * factor - g_star) * factor

    def bwd(G):
        return ps.soft_rdf_bwd(g, D, "all", dmin, sigma, 1.0, bins, G)

    def plain():
        gplain.build(X, T, "all", 2.0)
        ps.spatstat(gplain, D, "all", dmin, bins, [], rdf=True, out=plain_out, check=False)

    for _ in range(2):
        G = loss_grad(fwd())
        bwd(G)
        plain()
    torch.cuda.synchronize()
    reps = 3
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(reps)]
    for r in range(reps):
        ev[r][0].record()
        h = fwd()
        G = loss_grad(h)
        ev[r][1].record()
        bwd(G)
        ev[r][2].record()
        plain()
        ev[r][3].record()
    torch.cuda.synchronize()
    f_ms = sum(ev[r][0].elapsed_time(ev[r][1]) for r in range(reps)) / reps
    b_ms = sum(ev[r][1].elapsed_time(ev[r][2]) for r in range(reps)) / reps
    p_ms = sum(ev[r][2].elapsed_time(ev[r][3]) for r in range(reps)) / reps
    n_pairs = int(plain_out["meta"][1].item())
    g.close()
    gp.close()
    gplain.close()
    return {"workload": f"needle {N} ions (1e7 target), all-all, sigma=0.05 nm, r=[0,0.02,2] nm, d_srf>=2.3 nm",
            "n_central": int(n_c), "fwd_ms": f_ms, "bwd_ms": b_ms, "fwd_bwd_ms": f_ms + b_ms,
            "plain_exact_rdf_ms": p_ms, "fwd_bwd_over_plain": (f_ms + b_ms) / p_ms,
            "plain_pairs_per_s": n_pairs / (p_ms * 1e-3), "reps": reps,
            "cell_scale": args.soft_cell_scale,
            "timing": "CUDA events, eager, grid build included in fwd and plain; the plain exact RDF on half-size cells "
                      "in passes (its fastest form)"}


def measure_sdm(args, dev):
    """Spatial distribution maps on the 8.07e6-ion needle with the paper's strong-scaling setting
    (ROI radius 2 nm, cubic voxels of edge 0.025 nm: 160^3 voxels), d_srf >= 2 nm: Sc-Sc and
    all-all, each grid build + map against the plain exact RDF over the same pairs."""
    import torch

    import paper_2004_05188_gb300 as ps

    xyz, t, d = make_cloud("needle8m")
    N = xyz.shape[0]
    X = torch.from_numpy(xyz).to(dev)
    T = torch.from_numpy(t).to(dev)
    D = torch.from_numpy(d).to(dev)
    R, w, nv, dmin = 2.0, 0.025, 160, 2.0
    bins = (0.0, R, 1)
    g = ps.Grid(N)
    res = {"workload": f"needle {N} ions, ROI radius {R} nm, voxel {w} nm ({nv}^3), d_srf>={dmin} nm",
           "timing": "CUDA events, eager, grid build included, best of 3"}
    for name, types in (("Sc-Sc", [1]), ("all-all", "all")):
        out = ps.sdm(g.build(X, T, types, R), D, types, dmin, R, w, nv)
        plain_out = ps.spatstat(g, D, types, dmin, bins, [], rdf=True)

        def run_sdm():
            g.build(X, T, types, R)
            ps.sdm(g, D, types, dmin, R, w, nv, out=out)

        def run_plain():
            g.build(X, T, types, R)
            ps.spatstat(g, D, types, dmin, bins, [], rdf=True, out=plain_out, check=False)

        times = {}
        for key, fn in (("sdm", run_sdm), ("plain", run_plain)):
            fn()
            best = None
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
            times[key] = best
        meta = out["meta"].cpu().numpy()
        if meta[3] != 0 or int(meta[1]) != int(plain_out["meta"][1].item()):
            raise RuntimeError(f"SDM {name}: status {meta[3]} or pair count differs from the RDF")
        res[name] = {"n_central": int(meta[0]), "pairs": int(meta[1]), "sdm_ms": times["sdm"],
                     "plain_rdf_ms": times["plain"], "sdm_pairs_per_s": int(meta[1]) / (times["sdm"] * 1e-3),
                     "sdm_over_plain": times["sdm"] / times["plain"]}
    g.close()
    return res


def measure_cluster(args, dev):
    """Maximum-separation clustering of the Sc ions of the 8.07e6-ion needle over the paper's
    synthetic-benchmark sweep d_max = [0.10, 0.05, 0.70] nm (13 runs), N_min = 5; clusters whose
    ions all have d_srf >= 2 nm count as interior.  Each run = grid build + clustering."""
    import torch

    import paper_2004_05188_gb300 as ps

    xyz, t, d = make_cloud("needle8m")
    N = xyz.shape[0]
    X = torch.from_numpy(xyz).to(dev)
    T = torch.from_numpy(t).to(dev)
    D = torch.from_numpy(d).to(dev)
    d_maxes = [round(0.10 + 0.05 * i, 2) for i in range(13)]
    g = ps.Grid(N)
    out = None

    def run(dm):
        nonlocal out
        g.build(X, T, [1], dm * (1 + 1e-6))  # r_cut just above d_max: float32 r_cut^2 >= (float)(d_max^2)
        out = ps.cluster(g, D, dm, 5, 2.0, 1024, out=out)

    run(d_maxes[-1])
    torch.cuda.synchronize()
    rows = []
    total = 0.0
    for dm in d_maxes:
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run(dm)
            e1.record()
            torch.cuda.synchronize()
            best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
        m = out["meta"].cpu().numpy()
        if m[4] != 0:
            raise RuntimeError(f"clustering status {m[4]}")
        rows.append({"d_max": dm, "ms": round(best, 4), "clusters": int(m[1]), "ions_in_clusters": int(m[2]),
                     "interior_clusters": int(m[3])})
        total += best
    g.close()
    return {"workload": f"needle {N} ions, Sc ({int(m[0])} ions), d_max=[0.10,0.05,0.70] nm, N_min=5",
            "sweep_ms": total, "runs": rows, "timing": "CUDA events, eager, grid build included, best of 3 per run"}


def measure_batched(args, dev):
    """256 ROIs (needles and cylinders, log-uniform 1e4..1e7 ions), each with the sweep
    k = 1..20, r_max in {1, 2, 3} nm (0.01 nm bins), d_srf >= {0, 1, 2} nm, type pairs
    all-all, Sc-Sc, Al-Sc: one CUDA-graph replay of the batched path for all ROIs, against one
    plain exact call per ROI and sweep point (27 calls per ROI, each with k = 1..20) on all ROIs."""
    import torch

    import paper_2004_05188_gb300 as ps
    from paper_2004_05188_gb300 import specimen

    sizes = specimen.roi_sizes(args.batch_rois)
    t0 = time.perf_counter()
    host = [specimen.roi(i, n) for i, n in enumerate(sizes)]
    gen_s = time.perf_counter() - t0
    rois = [tuple(torch.from_numpy(a).to(dev) for a in r) for r in host]
    n_ions = int(sum(r[0].shape[0] for r in rois))
    del host
    bins, rmax, dsrf = (0.0, 0.01, 300), [100, 200, 300], [0.0, 1.0, 2.0]
    pairs, k_max = [("all", "all"), ([1], [1]), ([0], [1])], 20

    def graph_time(b, reps=1):
        out = torch.empty(b.shape, dtype=torch.int64, device=dev)
        b.run(out)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            b.run(out)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    sub = list(range(0, len(rois), max(1, len(rois) // 16)))[:16]
    # cell size of the batched kernel: the autotuner's choice on the subset
    from paper_2004_05188_gb300 import autotune

    cand = (args.batch_cell_scale,) if args.no_autotune else (1.0, 0.5)
    sub_t = {}
    for cs in cand:
        bs = ps.Batch([rois[i] for i in sub], bins, rmax, dsrf, pairs, k_max, cs)
        sub_t[(cs, 0)] = graph_time(bs)[0]
        bs.close()
    best_cs = autotune.choose(sub_t)[0]
    sub_ms = sub_t[(best_cs, 0)]
    b = ps.Batch(rois, bins, rmax, dsrf, pairs, k_max, best_cs)
    all_ms, out = graph_time(b)
    meta = out[..., -(4 + 2 * k_max):]
    n_central_all = int(meta[:, 0, -1, 0, 0].sum().item())  # all-all, r_max 3, d_srf >= 0
    b.close()
    del out

    ks = list(range(1, k_max + 1))
    # the plain path on all ROIs: one grid build per (ROI, pair, r_max) and one ps_spatstat per sweep point
    grid = ps.Grid(max(r[0].shape[0] for r in rois), best_cs)
    pouts = {nb: dict(rdf=torch.empty(nb, dtype=torch.int64, device=dev),
                      knn=torch.empty((k_max, nb), dtype=torch.int64, device=dev),
                      meta=torch.empty(4 + 2 * k_max, dtype=torch.int64, device=dev)) for nb in rmax}

    def plain(idx):
        for i in idx:
            X, T, D = rois[i]
            for ctr, nbr in pairs:
                for nb in rmax:
                    grid.build(X, T, nbr, nb * 0.01 * (1 + 1e-6))
                    for dmin in dsrf:
                        ps.spatstat(grid, D, ctr, dmin, (0.0, 0.01, nb), ks, out=pouts[nb], check=False)

    plain(sub)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plain(range(len(rois)))
    e1.record()
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    grid.close()
    return {"workload": f"{len(rois)} ROIs, {n_ions} ions (log-uniform 1e4..1e7), k=1..20, r_max {{1,2,3}} nm, "
                        "d_srf {0,1,2} nm, pairs all-all/Sc-Sc/Al-Sc",
            "sweep_points": len(rois) * 27, "batched_ms": all_ms, "plain_ms": plain_ms,
            "plain_over_batched": plain_ms / all_ms,
            "ion_queries_per_s": n_central_all / (all_ms * 1e-3), "cell_scale": best_cs,
            "autotune_subset_ms": {f"cell_scale={k[0]}": round(v, 2) for k, v in sub_t.items()},
            "host_generation_s": gen_s,
            "timing": "CUDA events; batched = one CUDA-graph replay for all ROIs (grid builds + one persistent "
                      "query kernel + expansion); plain = one eager grid build per (ROI, pair, r_max) and one "
                      "ps_spatstat per sweep point, all ROIs"}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
FAMS = ["reset", "select", "geometry", "count", "scan", "scatter", "central", "query", "knn_full", "rdf_sym",
        "epilogue"]
QUERY_FAMS = ("query", "knn_full", "rdf_sym")  # the pair tests: one pass, or the near kNN, fallback and RDF passes
BUILD_FAMS = ("select", "geometry", "count", "scan", "scatter", "central")


KERNEL_NAMES = {"query": "k_query_warp (one pass, or the near-radius kNN pass)",
                "knn_full": "k_query_warp (full-radius kNN fallback)", "rdf_sym": "k_rdf_sym (RDF over unordered pairs)"}


def rooflines(prof, st, steps, peaks, hbm_peak, hbm_src, traffic):
    """Roofline figures of one measurement: the dominant query kernel (by time) against the
    measured FP32 add/multiply throughput (its bound), every query pass the same way, the query
    against the measured shared-atomic rate (its RDF increments), and the build kernels against the
    measured HBM copy bandwidth.  prof: {family: (launches, ms)} summed over `steps` steps; st:
    per-step counts of every combination; traffic: stored_traffic(...) or None."""
    q_n = sum(prof[f][0] for f in QUERY_FAMS)
    q_ms = sum(prof[f][1] for f in QUERY_FAMS)
    cands = sum(c["candidates"] for c in st["combos"]) * steps
    pairs = sum(c["n_pairs_local"] for c in st["combos"]) * steps
    alu_peak = max(peaks["fp32_scalar_gops"], peaks["fp32_packed_gops"]) * 1e-3  # TFLOP/s
    alu = FLOPS_PER_CANDIDATE * cands / (q_ms * 1e-3) / 1e12 if q_ms > 0 else 0.0
    atom_rate = pairs / (q_ms * 1e-3) / 1e9 if q_ms > 0 else 0.0
    q_bytes = sum(algorithmic_bytes("query", st, c) for c in st["combos"]) * steps
    b_bytes = sum(algorithmic_bytes(f, st, c) for f in BUILD_FAMS for c in st["combos"]) * steps
    b_ms = sum(prof[f][1] for f in BUILD_FAMS)
    tot_ms = sum(v[1] for v in prof.values())

    def launching(fam):  # the combinations that launch this family's kernel once per step
        if fam == "query":
            return [c["name"] for c in st["combos"]]
        return [c["name"] for c in st["combos"] if c.get("split")]

    by_kernel = {}
    for fam in QUERY_FAMS:
        n, ms = prof[fam]
        if n == 0:
            continue
        tests = None if fam == "knn_full" else sum(c.get("candidates_by_pass", {}).get(fam, 0)
                                                     for c in st["combos"]) * steps
        tf = FLOPS_PER_CANDIDATE * tests / (ms * 1e-3) / 1e12 if tests is not None and ms > 0 else None
        rec = traffic["kernels"].get(fam) if traffic else None
        only_rec = traffic is not None and launching(fam) == [traffic["combination"]]
        by_kernel[fam] = {
            "kernel": KERNEL_NAMES[fam], "launches": n, "avg_launch_ms": ms / n,
            "flops_per_launch": FLOPS_PER_CANDIDATE * tests / n if tests is not None else None,
            "achieved_tflops": tf, "frac": tf / alu_peak if tf is not None and alu_peak > 0 else None,
            "traffic": rec if only_rec else None,
            "traffic_per_launch_of": (traffic["combination"] if rec is not None else None),
            "traffic_recorded": rec}
    dom = max(by_kernel, key=lambda f: prof[f][1]) if by_kernel else "query"
    d = by_kernel.get(dom, {})
    return {
        "bound": "alu", "kernel": KERNEL_NAMES[dom], "family": dom,
        "achieved": d.get("achieved_tflops") or 0.0, "peak": alu_peak, "unit": "TFLOP/s", "frac": d.get("frac"),
        "peak_source": f"measured: ps_measure_peaks FP32 add/multiply, {peaks['num_sms']} SMs at "
                       f"{peaks['sm_mhz']:.0f} MHz (scalar {peaks['fp32_scalar_gops']:.0f}, packed f32x2 "
                       f"{peaks['fp32_packed_gops']:.0f} Gop/s; the larger is the peak)",
        "traffic": d.get("traffic"),
        "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel, from the "
                        "stored ncu record (profiles/query_traffic.json) for these kernel sources, this workload "
                        "and this configuration; null if none",
        "algorithmic_bytes_per_launch": (algorithmic_bytes("query", st, next(c for c in st["combos"]
                                                                            if c["name"] == traffic["combination"]))
                                         if traffic and d.get("traffic") else None),
        "per_unit": f"{FLOPS_PER_CANDIDATE} FP32 operations per candidate test (3 sub, 3 mul, 2 add, 1 compare)",
        "flops_per_launch": d.get("flops_per_launch"), "launches": d.get("launches"),
        "avg_launch_ms": d.get("avg_launch_ms"),
        "by_kernel": by_kernel,
        "all_query_passes": {"achieved": alu, "frac": alu / alu_peak if alu_peak > 0 else None, "launches": q_n,
                             "avg_launch_ms": q_ms / max(1, q_n), "candidate_tests_per_step": cands // max(1, steps)},
        "pass_ms_per_step": {f: prof[f][1] / max(1, steps) for f in QUERY_FAMS},
        "timing": "CUDA events around every launch on the launching stream, inside the timed region",
        "time_share": q_ms / tot_ms if tot_ms > 0 else None,
        "shares": {k: round(v[1] / tot_ms, 5) for k, v in prof.items()} if tot_ms > 0 else None,
        "smem_atomic": {"achieved": atom_rate, "peak": peaks["smem_atomic_gops"], "unit": "G shared-atomic adds/s",
                        "frac": atom_rate / peaks["smem_atomic_gops"] if peaks["smem_atomic_gops"] > 0 else None,
                        "per_unit": "one 32-bit shared-memory increment per neighbour pair binned",
                        "peak_source": "measured: ps_measure_peaks, conflict-free 32-bit shared atomics"},
        "hbm_query": {"achieved": q_bytes / (q_ms * 1e-3) / 1e9 if q_ms > 0 else 0.0, "peak": hbm_peak,
                      "unit": "GB/s", "per_unit": "16 B per neighbour record + 16 B per central + 8 B per cell"},
        "hbm_build": {"achieved": b_bytes / (b_ms * 1e-3) / 1e9 if b_ms > 0 else 0.0, "peak": hbm_peak,
                      "unit": "GB/s", "frac": (b_bytes / (b_ms * 1e-3) / 1e9) / hbm_peak if b_ms > 0 else None,
                      "kernels": list(BUILD_FAMS), "ms_per_step": b_ms / max(1, steps),
                      "algorithmic_bytes_per_step": b_bytes / max(1, steps), "peak_source": hbm_src,
                      "by_kernel": {f: {"ms_per_step": prof[f][1] / max(1, steps),
                                        "gb_per_step": sum(algorithmic_bytes(f, st, c) for c in st["combos"]) / 1e9,
                                        "frac": (sum(algorithmic_bytes(f, st, c) for c in st["combos"]) * steps
                                                 / (prof[f][1] * 1e-3) / 1e9 / hbm_peak) if prof[f][1] > 0 else None}
                                    for f in BUILD_FAMS}},
    }


def combo_stats(ps, g, o, name, ctr, nbr, X, T, D, t_host, wl, stencil, split=False):
    """Counts of one combination after its build + query (reporting only, untimed).  candidates:
    the distance tests of the query -- one pass: every central against its stencil; in passes
    (split): every central against its near kNN block (its own 2 x 2 x 2 cells on half-size
    cells, the 27 cells around its cell on third-size cells) plus every unordered pair of records
    in each other's stencil once (symmetric RDF), the few full-radius fallback searches not
    counted."""
    meta = o["meta"].cpu().numpy()
    if meta[3] != 0:
        raise RuntimeError(f"device status {meta[3]} for {name}")
    info = g.info()
    mc, mn = ps.type_mask(ctr), ps.type_mask(nbr)
    lut = np.array([bool((int(mc[v >> 6]) >> (v & 63)) & 1) for v in range(256)])
    n_typed = sum(int(np.count_nonzero(lut[t_host[a:a + (1 << 26)]])) for a in range(0, t_host.shape[0], 1 << 26))
    subset = bool(np.all((mc & ~mn) == 0))
    cs = g.cell_scale
    if split and subset and stencil >= 2:
        if not wl["ks"]:
            near = 0
        elif stencil == 2:  # each central's own 2 x 2 x 2 block of cells
            near = octant_tests(X, T, D, ctr, nbr, wl["dsrf_min"], info)
        else:  # the 27 cells around the central's cell
            near = candidate_tests(X, T, D, ctr, nbr, wl["dsrf_min"], info, 1)
        full = candidate_tests(X, T, D, nbr, nbr, wl["dsrf_min"], info, stencil, all_records=True, cell_scale=cs)
        sym = (full - info["n_nbr"]) // 2
        by_pass = {"query": near, "rdf_sym": sym}
        cands = near + sym
    else:
        cands = candidate_tests(X, T, D, ctr, nbr, wl["dsrf_min"], info, stencil, cell_scale=cs)
        by_pass = {"query": cands}
    return dict(name=name, n_nbr=info["n_nbr"], n_cells=info["n_cells"], n_central=int(meta[0]),
                n_ctr_typed=n_typed, n_pairs_local=int(meta[1]), subset=subset, candidates=cands,
                candidates_by_pass=by_pass, split=bool(split and subset and stencil >= 2))


def e2e_runner(dev, stream, sets, hosts, step, outs, res_h):
    """End to end through the public API: every step copies its inputs from pinned host memory on a
    copy stream (into one of the device buffer sets, so that the copy of step k+1 overlaps the
    compute of step k when there are two sets), runs the step and reads the results back."""
    import torch

    copy_s = torch.cuda.Stream(device=dev)
    ev_copy = [torch.cuda.Event() for _ in sets]
    ev_used = [torch.cuda.Event() for _ in sets]

    def d2h():
        for o, h in zip(outs, res_h):
            for k in o:
                if o[k] is not None:
                    h[k].copy_(o[k], non_blocking=True)

    def run(n_steps):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        copy_s.wait_event(t0)
        for k in range(n_steps):
            b = k % len(sets)
            with torch.cuda.stream(copy_s):
                if k >= len(sets):
                    copy_s.wait_event(ev_used[b])
                for dst, src in zip(sets[b], hosts):
                    dst.copy_(src, non_blocking=True)
                ev_copy[b].record(copy_s)
            stream.wait_event(ev_copy[b])
            step(*sets[b])
            ev_used[b].record(stream)
            d2h()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    return run


def measure_sharded(args, wl_name, wl, dev, dist, world, rank, peaks):
    """The large needle, slab-sharded over the ranks (one slab at N = 1): eager steps with the
    library's per-launch events on, inside the timed region."""
    import torch

    import paper_2004_05188_gb300 as ps
    from paper_2004_05188_gb300 import shard, specimen

    bins = wl["bins"]
    r_cut = float(np.float32(bins[0] + bins[1] * bins[2]))
    p = needle_params(wl_name)
    t0 = time.perf_counter()
    counts = specimen.needle_plan(p)
    cuts = shard.layer_cuts(counts, world)
    halo = shard.halo_layers(p.a, r_cut, p.sig_z)
    pinned = []

    def alloc(n):
        bufs = (torch.empty((n, 3), dtype=torch.float32, pin_memory=True),
                torch.empty(n, dtype=torch.uint8, pin_memory=True),
                torch.empty(n, dtype=torch.float32, pin_memory=True))
        pinned.extend(bufs)
        return tuple(b.numpy() for b in bufs)

    xyz, t, d, core = shard.slab_needle(p, counts, cuts, rank, halo, alloc)
    gen_s = time.perf_counter() - t0
    Xh, Th, Dh = pinned
    N = xyz.shape[0]
    X = torch.empty((N, 3), dtype=torch.float32, device=dev)
    T = torch.empty(N, dtype=torch.uint8, device=dev)
    D = torch.empty(N, dtype=torch.float32, device=dev)
    for dst, src in zip((X, T, D), (Xh, Th, Dh)):
        dst.copy_(src, non_blocking=True)
    torch.cuda.synchronize()

    # cell size for the grid shared by the combinations: the autotuner's choice for the dominant
    # combination, timed on a contiguous z-slice of the local cloud (1/32 of it; untimed)
    name0, ctr0, nbr0 = wl["combos"][0]
    from paper_2004_05188_gb300 import autotune

    a = N // 2 - N // 64
    b = a + N // 32
    if args.no_autotune:
        tuned = {"cell_scale": args.cell_scale, "dense_min": args.dense_min, "split": int(args.split),
                 "timings_ms": None}
    else:
        tuned = autotune.tune(X[a:b], T[a:b], D[a:b], nbr0, ctr0, wl["dsrf_min"], bins, wl["ks"],
                              candidates=((1.0, 0), (0.5, 0), (0.5, 0, 1), (1 / 3, 0, 1), (1.0, 128)), reps=2)
    cs, dm, sp = tuned["cell_scale"], tuned["dense_min"], int(tuned.get("split", 0))
    # the other combinations keep the cell size (one grid) and tune only the query options
    qopts = {name0: (dm, sp)}
    tunings = {name0: tuned.get("timings_ms")}
    for name, ctr, nbr in wl["combos"][1:]:
        if args.no_autotune or cs >= 1.0:
            qopts[name] = (dm, sp if cs < 1.0 else 0)
            continue
        t2 = autotune.tune(X[a:b], T[a:b], D[a:b], nbr, ctr, wl["dsrf_min"], bins, wl["ks"],
                           candidates=((cs, 0, 0), (cs, 0, 1)), reps=2)
        qopts[name] = (int(t2["dense_min"]), int(t2.get("split", 0)))
        tunings[name] = t2.get("timings_ms")
    if dist is not None:  # every rank uses rank 0's choice (results do not depend on it; timings would)
        pick = [(cs, dm, sp, qopts, tunings)]
        dist.broadcast_object_list(pick, src=0)
        cs, dm, sp, qopts, tunings = pick[0]
    grid = ps.Grid(N, cs, dm, bool(sp))
    nk = len(wl["ks"])
    outs = [dict(rdf=torch.empty(bins[2], dtype=torch.int64, device=dev),
                 knn=torch.empty((nk, bins[2]), dtype=torch.int64, device=dev),
                 meta=torch.empty(ps.META_HEAD + 2 * nk, dtype=torch.int64, device=dev)) for _ in wl["combos"]]
    stream = torch.cuda.current_stream()

    def step(Xs=X, Ts=T, Ds=D):
        for (name, ctr, nbr), o in zip(wl["combos"], outs):
            grid.set_query_opts(*qopts[name])
            grid.build(Xs, Ts, nbr, r_cut)
            ps.spatstat(grid, Ds, ctr, wl["dsrf_min"], bins, wl["ks"], out=o, check=False)
        for o in outs:
            shard.combine(dist, o)

    # one verified pass per combination (device status, local counts for the rooflines)
    st = {"n_ions": N, "combos": []}
    stencil = grid.stencil
    for (name, ctr, nbr), o in zip(wl["combos"], outs):
        grid.set_query_opts(*qopts[name])
        grid.build(X, T, nbr, r_cut)
        ps.spatstat(grid, D, ctr, wl["dsrf_min"], bins, wl["ks"], out=o, check=False)
        torch.cuda.synchronize()
        st["combos"].append(combo_stats(ps, grid, o, name, ctr, nbr, X, T, D, t, wl, stencil, bool(qopts[name][1])))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    n_queries = sum(int(o["meta"][0].item()) for o in outs)  # every rank's centrals (after the combine)
    n_pairs = sum(int(o["meta"][1].item()) for o in outs)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sampler = ClockSampler(gpu_index(dev.index), args.clocks_csv if rank == 0 else None)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ps.prof_enable(FAMS)
    sampler.start()
    barrier(dist)
    torch.cuda.synchronize()
    lc0 = ps.launch_count()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (not timed)
        ev0[k].record(stream)
        step()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    wall = time.perf_counter() - wall0
    launches = ps.launch_count() - lc0
    clocks = sampler.stop()
    prof = {f: ps.prof_read(f) for f in FAMS}
    ps.prof_enable([])
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    T_ms, _ = rank_reduce(dist, dev, float(sum(step_ms)), [])
    value = n_queries * args.steps / (T_ms * 1e-3)

    e2e = None
    if not args.no_e2e:
        res_h = [{k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in o.items()} for o in outs]
        sets = [(X, T, D)]
        free = torch.cuda.mem_get_info(dev)[0]
        if free > X.nbytes + T.nbytes + D.nbytes + (8 << 30):  # a second input set: copies overlap compute
            sets.append((torch.empty_like(X), torch.empty_like(T), torch.empty_like(D)))
        run = e2e_runner(dev, stream, sets, (Xh, Th, Dh), step, outs, res_h)
        run(len(sets))
        E_ms, _ = rank_reduce(dist, dev, run(args.steps), [])
        h2d = Xh.nbytes + Th.nbytes + Dh.nbytes
        d2h = sum(v.numel() * v.element_size() for o in outs for v in o.values())
        e2e = {"value": n_queries * args.steps / (E_ms * 1e-3), "unit": "ion-queries/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": E_ms / args.steps, "steps": args.steps,
               "mode": (f"{len(sets)} device input set(s): " +
                        ("the H2D of step k+1 overlaps the compute of step k" if len(sets) > 1 else
                         "H2D, compute and D2H in sequence"))}
        del sets, res_h

    hbm_peak, hbm_src = load_hbm_peak()
    kcfg = {name: {"cell_scale": float(cs), "dense_min": int(qopts[name][0]), "split": int(qopts[name][1])}
            for name, _, _ in wl["combos"]}
    import hashlib

    dig = hashlib.sha256()
    for o in outs:  # the whole specimen's histograms and counters (after the combine)
        for k in ("rdf", "knn", "meta"):
            dig.update(o[k].cpu().numpy().tobytes())
    roof = rooflines(prof, st, args.steps, peaks, hbm_peak, hbm_src, stored_traffic(wl_name, kcfg))
    grid.close()
    res = {"value": value, "T_ms": T_ms, "n_queries": n_queries, "n_pairs": n_pairs, "launches": launches,
           "clocks": clocks, "wall": wall, "e2e": e2e, "roofline": roof, "n_ions_local": N,
           "kernel_config": kcfg, "autotune": tunings, "generation_s": gen_s,
           "slab": {"layers": [int(cuts[rank]), int(cuts[rank + 1])], "halo_layers": halo, "ions_generated": N,
                    "core_ions": int(core[1] - core[0])},
           "step_ms_min_max": [min(step_ms), max(step_ms)], "result_sha256": dig.hexdigest()}
    del X, T, D, pinned, Xh, Th, Dh
    torch.cuda.empty_cache()
    return res


def measure_replica(args, wl_name, wl, dev, dist, world, rank, peaks, steps, warmup, do_e2e):
    """A small workload, one independent specimen per rank: each step captured once in a CUDA
    graph and replayed; the per-launch timing comes from an eager pass with the library's
    per-launch events (the combinations one after the other, so that every launch is timed alone)."""
    import torch

    import paper_2004_05188_gb300 as ps

    cloud = make_cloud(wl_name, seed_offset=1000 * rank)
    xyz, t, d = cloud
    N = xyz.shape[0]
    X, T, D = (torch.from_numpy(a).to(dev) for a in (xyz, t, d))
    bins = wl["bins"]
    r_cut = float(np.float32(bins[0] + bins[1] * bins[2]))
    tuned = {}
    for name, ctr, nbr in wl["combos"]:
        if args.no_autotune:
            tuned[name] = {"cell_scale": args.cell_scale, "dense_min": args.dense_min, "split": int(args.split)}
        else:
            from paper_2004_05188_gb300 import autotune

            tuned[name] = autotune.tune(X, T, D, nbr, ctr, wl["dsrf_min"], bins, wl["ks"])
    grids = [ps.Grid(N, tuned[name]["cell_scale"], tuned[name]["dense_min"], bool(tuned[name].get("split", 0)))
             for name, _, _ in wl["combos"]]
    nk = len(wl["ks"])
    outs = [dict(rdf=torch.empty(bins[2], dtype=torch.int64, device=dev),
                 knn=torch.empty((nk, bins[2]), dtype=torch.int64, device=dev),
                 meta=torch.empty(ps.META_HEAD + 2 * nk, dtype=torch.int64, device=dev)) for _ in wl["combos"]]
    stream = torch.cuda.current_stream()
    combo_streams = None
    if len(wl["combos"]) > 1 and not args.serial_combos:
        # the type combinations are independent analyses: each on its own stream, so that the
        # short, latency-bound kernels of one overlap with the other's
        combo_streams = [torch.cuda.Stream(device=dev) for _ in wl["combos"]]

    def step(Xs=X, Ts=T, Ds=D, serial=False):
        if combo_streams is None or serial:
            for (name, ctr, nbr), g, o in zip(wl["combos"], grids, outs):
                g.build(Xs, Ts, nbr, r_cut)
                ps.spatstat(g, Ds, ctr, wl["dsrf_min"], bins, wl["ks"], out=o, check=False)
            return
        cur = torch.cuda.current_stream()
        for cs in combo_streams:
            cs.wait_stream(cur)
        for (name, ctr, nbr), g, o, cs in zip(wl["combos"], grids, outs, combo_streams):
            with torch.cuda.stream(cs):
                g.build(Xs, Ts, nbr, r_cut)
                ps.spatstat(g, Ds, ctr, wl["dsrf_min"], bins, wl["ks"], out=o, check=False)
        for cs in combo_streams:
            cur.wait_stream(cs)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    step()
    torch.cuda.synchronize()
    st = {"n_ions": N, "combos": []}
    for (name, ctr, nbr), g, o in zip(wl["combos"], grids, outs):
        stencil = g.stencil
        st["combos"].append(combo_stats(ps, g, o, name, ctr, nbr, X, T, D, t, wl, stencil,
                                        bool(tuned[name].get("split", 0))))
    n_queries = sum(c["n_central"] for c in st["combos"])
    n_pairs = sum(c["n_pairs_local"] for c in st["combos"])
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ps.prof_enable(FAMS)
    for _ in range(steps):
        flush.zero_()
        step(serial=True)
    torch.cuda.synchronize()
    prof = {f: ps.prof_read(f) for f in FAMS}
    ps.prof_enable([])
    lc = ps.launch_count()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    kernels_per_step = ps.launch_count() - lc
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_index(dev.index), None)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    sampler.start()
    barrier(dist)
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev0[k].record(stream)
        graph.replay()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop()
    T_ms, (tot_q, tot_p) = rank_reduce(dist, dev, float(sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))),
                                       [n_queries, n_pairs])
    e2e = None
    if do_e2e:
        Xh, Th, Dh = (torch.from_numpy(a).pin_memory() for a in (xyz, t, d))
        res_h = [{k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in o.items()} for o in outs]
        XB, TB, DB = torch.empty_like(X), torch.empty_like(T), torch.empty_like(D)
        graph_b = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_b):
            step(XB, TB, DB)
        graphs = {X.data_ptr(): graph, XB.data_ptr(): graph_b}
        run = e2e_runner(dev, stream, [(X, T, D), (XB, TB, DB)], (Xh, Th, Dh),
                         lambda Xs, Ts, Ds: graphs[Xs.data_ptr()].replay(), outs, res_h)
        run(4)
        E_ms, _ = rank_reduce(dist, dev, run(steps), [])
        e2e = {"value": tot_q * steps / (E_ms * 1e-3), "unit": "ion-queries/s",
               "h2d_bytes_per_step": xyz.nbytes + t.nbytes + d.nbytes,
               "d2h_bytes_per_step": sum(v.numel() * v.element_size() for o in outs for v in o.values()),
               "ms_per_step": E_ms / steps,
               "mode": "pipelined: the H2D of step k+1 overlaps the compute of step k (two input buffer sets)"}
    hbm_peak, hbm_src = load_hbm_peak()
    kcfg = {name: {"cell_scale": float(tuned[name]["cell_scale"]), "dense_min": int(tuned[name]["dense_min"]),
                   "split": int(tuned[name].get("split", 0))} for name, _, _ in wl["combos"]}
    roof = rooflines(prof, st, steps, peaks, hbm_peak, hbm_src, stored_traffic(wl_name, kcfg))
    roof["timing"] = ("CUDA events around every launch on the launching stream, in an eager pass of the step with "
                      "the combinations one after the other (the timed steps are graph replays)")
    for g in grids:
        g.close()
    return {"value": tot_q * steps / (T_ms * 1e-3), "T_ms": T_ms, "n_queries": n_queries, "n_pairs": n_pairs,
            "launches": kernels_per_step * steps, "clocks": clocks, "e2e": e2e, "roofline": roof,
            "kernel_config": kcfg, "autotune": {k: v.get("timings_ms") for k, v in tuned.items()},
            "workload": wl["desc"], "n_ions": N, "ms_per_step": T_ms / steps, "steps": steps,
            "neighbour_pairs_per_s": tot_p * steps / (T_ms * 1e-3)}


def rank_reduce(dist, device, t_max, sums):
    """Whole-job numbers across ranks: the slowest rank's time and the summed counts.

    dist is torch.distributed (or None for one process); device is where the reduction
    tensors live (a CUDA device under NCCL, the CPU under gloo)."""
    import torch

    if dist is None:
        return float(t_max), [float(x) for x in sums]
    if dist.get_backend() == "gloo":
        device = "cpu"
    tt = torch.tensor([float(t_max)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ss = torch.tensor([float(x) for x in sums], dtype=torch.float64, device=device)
    dist.all_reduce(ss)
    return float(tt.item()), [float(x) for x in ss.tolist()]


def barrier(dist):
    if dist is not None:
        dist.barrier()


def local_rank() -> int:
    return int(os.environ.get("LOCAL_RANK", "0"))


def gpu_index(local: int) -> int:
    """nvidia-smi index of the GPU this rank uses (ranks that share a GPU share its index)."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = vis.split(",")
        return int(ids[local % len(ids)])
    return local


def run_gpu(args, wl_name, wl):
    import torch

    import paper_2004_05188_gb300 as ps

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = local_rank() % max(1, torch.cuda.device_count())
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        # NCCL, one GPU per rank; PS_BENCH_BACKEND=gloo combines through the host instead (ranks
        # that share a GPU: every rank's kernels are its own, only the host-side sum joins them)
        backend = os.environ.get("PS_BENCH_BACKEND", "nccl")
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    dev = torch.device("cuda", local)
    peaks = ps.measure_peaks()

    if wl.get("sharded"):
        head = measure_sharded(args, wl_name, wl, dev, dist, world, rank, peaks)
        scaling = "strong"
        parallelism = (f"z-slabs of equal ion count x{world} (r_cut halo each), one int64 sum all-reduce of the "
                       f"histograms per combination" if world > 1 else "one GPU, one slab (the whole specimen)")
    else:
        head = measure_replica(args, wl_name, wl, dev, dist, world, rank, peaks, args.steps, args.warmup,
                               not args.no_e2e)
        scaling = "weak"
        parallelism = f"replicas x{world} (independent specimens, no collective)"

    secondary = None
    if rank == 0 and world == 1 and not args.no_secondary and wl.get("sharded"):
        secondary = {}
        for name in SECONDARY:
            w2 = resolve(name)
            r = measure_replica(args, name, w2, dev, None, 1, 0, peaks, 20, 5, False)
            secondary[name] = {k: r[k] for k in ("workload", "value", "ms_per_step", "steps", "n_queries",
                                                 "neighbour_pairs_per_s", "kernel_config", "autotune", "clocks")}
            secondary[name]["roofline"] = {k: r["roofline"][k] for k in ("kernel", "achieved", "peak", "unit", "frac",
                                                                         "traffic", "avg_launch_ms", "time_share")}
            secondary[name]["roofline"]["all_query_passes_frac"] = r["roofline"]["all_query_passes"]["frac"]
            secondary[name]["smem_atomic_frac"] = r["roofline"]["smem_atomic"]["frac"]
            secondary[name]["hbm_build_frac"] = r["roofline"]["hbm_build"]["frac"]

    forms = None
    if rank == 0 and not args.no_forms:
        forms = {"soft": measure_soft(args, dev)}
        if args.batch_rois > 0:
            forms["batched"] = measure_batched(args, dev)
        forms["sdm"] = measure_sdm(args, dev)
        forms["cluster"] = measure_cluster(args, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        cloud = None if wl.get("sharded") else make_cloud(wl_name)
        orc, parts, pool, nq, desc = oracle_sampled(wl_name, wl, cores, target_s=3.0, cloud=cloud)
        reps, dt = 0, 0.0
        while reps < 3 or dt < 10.0:
            nq, t1 = oracle_steps(orc, parts, pool, wl, 1)
            reps += 1
            dt += t1
            if dt > 30.0:
                break
        pool.shutdown()
        cpu = {"value": nq * reps / dt, "unit": "ion-queries/s", "cores": cores, "kind": "oracle",
               "sample": f"{desc}; {nq} centrals per run, {reps} runs"}

    if rank == 0:
        line = {
            "metric": "ion-queries/s (exact kNN+RDF)", "value": head["value"], "unit": "ion-queries/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["T_ms"] / args.steps,
            "higher_is_better": True, "scaling": scaling, "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "n_ions": int(head.get("n_ions", head.get("n_ions_local", 0))),
                       "centrals_per_step": head["n_queries"], "neighbour_pairs_per_step": head["n_pairs"],
                       "kernel_config": head["kernel_config"], "autotune": head["autotune"],
                       "l2": "flushed between steps (512 MB write); the inputs also exceed L2",
                       "parallelism": parallelism},
            "neighbour_pairs_per_s": head["n_pairs"] * args.steps / (head["T_ms"] * 1e-3),
            "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": head["e2e"], "gpu_launches": head["launches"],
            "gpu_launches_per_step": head["launches"] / args.steps, "clocks": head["clocks"],
            "measured_peaks": peaks, "secondary": secondary, "forms": forms,
        }
        for k in ("slab", "generation_s", "step_ms_min_max", "result_sha256"):
            if k in head:
                line["config" if k == "slab" else k] = ({**line["config"], "slab_rank0": head[k]} if k == "slab"
                                                         else head[k])
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def resolve(name):
    wl = dict(WORKLOADS[name])
    r0, dr, stop = wl["spec"]
    wl["bins"] = (r0, dr, int(round((stop - r0) / dr)))
    return wl


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="needle2g", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--clocks-csv", default=None, help="file for the raw nvidia-smi clock samples of the timed region "
                                                         "(default: a temporary file)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serial-combos", action="store_true", help="small workloads: run the type combinations one "
                    "after the other on one stream (default: one stream each)")
    ap.add_argument("--no-forms", action="store_true", help="skip the smoothed-RDF, batched, SDM and clustering forms")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 8e6-needle and 2e5-cylinder figures")
    ap.add_argument("--batch-rois", type=int, default=256, help="ROIs of the batched measurement (0 skips it)")
    ap.add_argument("--batch-cell-scale", type=float, default=1.0)
    ap.add_argument("--soft-cell-scale", type=float, default=0.5, help="cell edge / r_cut of the smoothed-RDF grids")
    ap.add_argument("--cell-scale", type=float, default=1.0, help="cell edge / r_cut (>= 1/3)")
    ap.add_argument("--dense-min", type=int, default=0, help="centrals per cell for the staged CTA kernel (0: never)")
    ap.add_argument("--split", action="store_true", help="the query in passes (with --no-autotune; ps_grid_opts.split)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --cell-scale/--dense-min/--split instead of the autotuner")
    ap.add_argument("--only-form", choices=["soft", "batched", "sdm", "cluster"],
                    help="measure only this form (no exact step line)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    wl = resolve(args.workload)
    if args.impl == "reference":
        return run_reference(args, args.workload, wl)
    import __graft_entry__

    __graft_entry__.build()
    if args.only_form:
        import torch

        dev = torch.device("cuda", local_rank())
        torch.cuda.set_device(dev)
        fn = {"soft": measure_soft, "batched": measure_batched, "sdm": measure_sdm,
              "cluster": measure_cluster}[args.only_form]
        print(json.dumps({"form": args.only_form, **fn(args, dev)}), flush=True)
        return 0
    return run_gpu(args, args.workload, wl)


if __name__ == "__main__":
    sys.exit(main())
