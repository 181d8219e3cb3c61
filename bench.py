#!/usr/bin/env python
"""Benchmark of the exact kNN + RDF spatial-statistics path on one GB300.

Default workload: the ~8.07e6-ion needle (tip radius 20 nm, half-angle
10 deg, height 100 nm, 30 ions/nm^3, Al3Sc precipitates), type combinations
Sc-Sc and Si-Si, k in {1, 5, 10}, RDF on r = [0, 0.01, 2] nm, central ions
with d_srf >= 2 nm.  One step = for each combination: build the neighbour
cell grid (binner) and run the kNN + RDF query (central list + query
kernel), i.e. every step of the exact path, with inputs resident in HBM.

value   = ion queries (central ions evaluated, summed over the combinations
          and over ranks) per second of device time.
e2e     = the same metric through the public Python API with the inputs in
          pinned host memory: H2D copy + both combinations + D2H of results.
roofline: the dominant kernel family, timed with CUDA events on its stream
          in the timed region, against the measured HBM copy bandwidth.
cpu_baseline: the oracle (C) on a bounded z-slab sample, on every host core (one
          z-slab of centrals per thread, exact sum), and on one core.

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
    "needle8m": dict(
        desc="needle 8.07e6 ions (r_tip 20 nm, 10 deg, h 100 nm, 30/nm^3, Al3Sc precipitates); Sc-Sc + Si-Si; "
             "kNN k=1,5,10 + RDF r=[0,0.01,2] nm; d_srf>=2 nm",
        combos=[("Sc-Sc", [1], [1]), ("Si-Si", [2], [2])], ks=[1, 5, 10], spec=(0.0, 0.01, 2.0), dsrf_min=2.0),
    "needle2g": dict(
        desc="needle 2e9 ions (r_tip 40 nm, 15 deg, h 812.6 nm, 30/nm^3, Al3Sc precipitates); all-all + Sc-Sc; "
             "kNN k=10 + RDF r=[0,0.01,2] nm; d_srf>=2 nm",
        combos=[("all-all", "all", "all"), ("Sc-Sc", [1], [1])], ks=[10], spec=(0.0, 0.01, 2.0), dsrf_min=2.0),
    "cylinder200k": dict(
        desc="Poisson cylinder 2e5 ions (R 10 nm, H 15.9 nm, 40/nm^3); all-all; kNN k=1 + RDF r=[0,0.01,2] nm; "
             "d_srf>=1 nm",
        combos=[("all-all", "all", "all")], ks=[1], spec=(0.0, 0.01, 2.0), dsrf_min=1.0),
}


def make_cloud(name: str, seed_offset: int = 0):
    from paper_2004_05188_gb300 import specimen

    if name == "needle8m":
        return specimen.needle(specimen.needle_8m_params(seed=2 + seed_offset))
    if name == "cylinder200k":
        return specimen.cylinder_small(seed=1 + seed_offset)
    if name == "needle2g":
        return specimen.needle(specimen.needle_2g_params(seed=5 + seed_offset))
    raise ValueError(name)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# FP32 pipe: 152 SMs x 128 lanes, one non-fused FP32 operation per lane per clock
N_SM, FP32_LANES = 152, 128
FLOPS_PER_CANDIDATE = 9  # d2 = ((dx*dx) + (dy*dy)) + (dz*dz): 3 sub, 3 mul, 2 add; 1 compare against the range


def alu_peak_tflops():
    """FP32 (non-FMA) peak from the unit counts and the maximum SM clock."""
    mhz = 2070.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return N_SM * FP32_LANES * mhz * 1e6 / 1e12, mhz


def query_sources_sha256() -> str:
    """Digest of the query kernels' sources: a stored ncu traffic figure holds only for this source."""
    import hashlib

    h = hashlib.sha256()
    for f in ("ps_query.cu", "ps_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2004_05188_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def stored_traffic(workload: str, kernel_config: dict):
    """DRAM bytes per query launch from the committed ncu summary, or None when that summary was
    taken on other kernel sources, another workload or another kernel configuration."""
    p = os.path.join(ROOT, "profiles", "query_traffic_needle8m.md")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        for line in f:
            if line.startswith("record: "):
                rec = json.loads(line[len("record: "):])
                if (rec.get("workload") == workload and rec.get("source_sha256") == query_sources_sha256()
                        and rec.get("kernel_config") == kernel_config):
                    return float(rec["dram_bytes_per_launch"])
    return None


def candidate_tests(X, T, D, ctr, nbr, dsrf_min, info, stencil):
    """Central x candidate tests one query makes on this grid: for every central, the neighbour
    records in the (2*stencil+1)^3 cells around its cell (clipped at the grid's faces).
    Counted with plain torch ops from the grid geometry (reporting only, untimed)."""
    import torch

    import paper_2004_05188_gb300 as ps

    def lut(types):
        m = ps.type_mask(types)
        return torch.tensor([bool((int(m[t >> 6]) >> (t & 63)) & 1) for t in range(256)], device=T.device)

    dims = info["dims"]
    org = torch.tensor(info["origin"], dtype=torch.float32, device=X.device)
    inv_h = float(np.float32(1.0 / float(info["cell"])))

    def cells(P):
        u = torch.floor((P - org) * inv_h).to(torch.int64)
        for a in range(3):
            u[:, a].clamp_(0, dims[a] - 1)
        return (u[:, 2] * dims[1] + u[:, 1]) * dims[0] + u[:, 0]

    Tl = T.long()
    cnt = torch.bincount(cells(X[lut(nbr)[Tl]]), minlength=info["n_cells"]).view(dims[2], dims[1], dims[0])
    s = int(stencil)
    for ax in range(3):  # box sum of width 2s+1 along each axis (exact, int64)
        c = torch.cumsum(torch.nn.functional.pad(cnt.movedim(ax, -1), (s + 1, s)), dim=-1)
        cnt = (c[..., 2 * s + 1:] - c[..., : -(2 * s + 1)]).movedim(-1, ax)
    cm = lut(ctr)[Tl] & (D >= dsrf_min)
    return int(cnt.reshape(-1)[cells(X[cm])].sum().item())


# ---------------------------------------------------------------------------
# clocks sampling during the timed region
# ---------------------------------------------------------------------------
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
def slab_sample(xyz, t, d, frac: float, halo: float):
    """A z-slab holding `frac` of the z-extent: its ions plus a halo of neighbours; halo ions are not central."""
    z = xyz[:, 2]
    zlo, zhi = float(z.min()), float(z.max())
    z0 = zlo + 0.5 * (zhi - zlo) * (1.0 - frac)
    z1 = z0 + frac * (zhi - zlo)
    keep = (z >= z0 - halo) & (z < z1 + halo)
    core = (z >= z0) & (z < z1)
    ds = np.where(core[keep], d[keep], np.float32(-1e30)).astype(np.float32)
    return xyz[keep], t[keep], ds


def oracle_step(orc, cloud, wl):
    xyz, t, d = cloud
    r0, dr, nb = wl["bins"]
    n = 0
    for _, ctr, nbr in wl["combos"]:
        r = orc.spatstat(xyz, t, d, ctr, nbr, wl["dsrf_min"], r0, dr, nb, wl["ks"])
        n += r["n_central"]
    return n


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def slab_parts(xyz, t, d, frac: float, halo: float, parts: int):
    """The z-slab of slab_sample split into `parts` consecutive z-slabs of centrals, each with its own
    halo of neighbours: independent oracle runs over them add up to the whole slab's exact counts."""
    z = xyz[:, 2]
    zlo, zhi = float(z.min()), float(z.max())
    z0 = zlo + 0.5 * (zhi - zlo) * (1.0 - frac)
    z1 = z0 + frac * (zhi - zlo)
    cuts = [z0 + (z1 - z0) * i / parts for i in range(parts + 1)]
    out = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        keep = (z >= a - halo) & (z < b + halo)
        core = (z >= a) & (z < b)
        out.append((xyz[keep], t[keep], np.where(core[keep], d[keep], np.float32(-1e30)).astype(np.float32)))
    return out


def oracle_step_parts(orc, parts, wl, pool):
    """One step of the oracle on every part, one host thread each (ctypes releases the GIL; the
    oracle keeps no global state)."""
    return sum(pool.map(lambda c: oracle_step(orc, c, wl), parts))


def oracle_sample_parallel(wl, cloud, pool, cores: int, target_s=1.0):
    """Bounded sample for the oracle on `cores` host threads: a z-slab, split in `cores` parts,
    whose parallel run takes ~target_s."""
    import oracle as orc

    orc.build()
    xyz, t, d = cloud
    halo = wl["bins"][1] * wl["bins"][2]
    frac = min(1.0, 0.02 * cores)
    while True:
        parts = slab_parts(xyz, t, d, frac, halo, cores)
        t0 = time.perf_counter()
        nq = oracle_step_parts(orc, parts, wl, pool)
        dt = time.perf_counter() - t0
        if dt >= 0.25 * target_s or frac >= 1.0:
            break
        frac = min(1.0, frac * max(2.0, 0.5 * target_s / max(dt, 1e-3)))
    return orc, parts, frac, nq, dt


def oracle_sample(wl_name, wl, cloud, target_s=1.0):
    """Bounded sample of the workload for the oracle: a z-slab whose single-threaded run takes ~target_s."""
    import oracle as orc

    xyz, t, d = cloud
    frac = 0.02
    while True:
        samp = slab_sample(xyz, t, d, frac, wl["bins"][1] * wl["bins"][2])
        t0 = time.perf_counter()
        nq = oracle_step(orc, samp, wl)
        dt = time.perf_counter() - t0
        if dt >= 0.25 * target_s or frac >= 1.0:
            break
        frac = min(1.0, frac * max(2.0, 0.5 * target_s / max(dt, 1e-3)))
    return orc, samp, frac, nq, dt


def run_reference(args, wl_name, wl):
    import concurrent.futures as cf

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cloud = make_cloud(wl_name)
    cores = host_cores()
    with cf.ThreadPoolExecutor(max_workers=cores) as pool:
        orc, parts, frac, nq, _ = oracle_sample_parallel(wl, cloud, pool, cores, target_s=1.0)
        for _ in range(args.warmup):
            oracle_step_parts(orc, parts, wl, pool)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            nq = oracle_step_parts(orc, parts, wl, pool)
            times.append(time.perf_counter() - t0)
    T = sum(times)
    v = nq * args.steps / T
    line = {
        "impl": "reference", "metric": "ion-queries/s (exact kNN+RDF)", "value": v, "unit": "ion-queries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["desc"], "sample": f"z-slab with {frac:.3f} of the height (+2 nm halo), "
                                                        f"split in {cores} slabs of centrals, one host thread each"},
        "cpu_baseline": {"value": v, "unit": "ion-queries/s", "cores": cores, "kind": "oracle",
                         "sample": f"z-slab {frac:.3f} of the height in {cores} slabs (+2 nm halo each), "
                                   f"{nq} centrals per step"},
        "e2e": {"value": v, "unit": "ion-queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def algorithmic_bytes(kid: str, st: dict) -> float:
    """Bytes the kernel family must move per step (reads + writes of its role), summed over the combinations."""
    N = st["n_ions"]
    tot = 0.0
    for c in st["combos"]:
        nn, nc, cells, ntm = c["n_nbr"], c["n_central"], c["n_cells"], c["n_ctr_typed"]
        if kid == "select":
            tot += N * 1 + nn * 12 + nn * 4
        elif kid == "central":
            tot += cells * 4 + N * 1 + ntm * 4 + nc * 12 + nc * 12
        elif kid == "count":
            tot += nn * (4 + 12 + 8)
        elif kid == "scatter":
            tot += nn * (4 + 8 + 12 + 4 + 16) + nc * (4 + 8 + 12 + 4 + 16)
        elif kid == "scan":
            tot += 2 * cells * (4 + 4 + 4 + 4)
        elif kid == "geometry":
            tot += cells * 4
        elif kid == "query":
            tot += nn * 16 + nc * 16 + 2 * cells * 4
    return tot


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
    g = ps.Grid(N)
    gp = ps.Grid(N)
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
        g.build(X, T, "all", 2.0)
        ps.spatstat(g, D, "all", dmin, bins, [], rdf=True, out=plain_out, check=False)

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
    return {"workload": f"needle {N} ions (1e7 target), all-all, sigma=0.05 nm, r=[0,0.02,2] nm, d_srf>=2.3 nm",
            "n_central": int(n_c), "fwd_ms": f_ms, "bwd_ms": b_ms, "fwd_bwd_ms": f_ms + b_ms,
            "plain_exact_rdf_ms": p_ms, "fwd_bwd_over_plain": (f_ms + b_ms) / p_ms,
            "plain_pairs_per_s": n_pairs / (p_ms * 1e-3), "reps": reps,
            "timing": "CUDA events, eager, grid build included in fwd and plain"}


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
    all-all, Sc-Sc, Al-Sc: one CUDA-graph replay of the batched path for all ROIs; and, on a
    subset of 16 ROIs spread over the size range, the batched path against one plain exact
    call per ROI and sweep point (27 calls per ROI, each with k = 1..20)."""
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
    grids = {i: ps.Grid(rois[i][0].shape[0], best_cs) for i in sub}

    def plain_all():
        for i in sub:
            X, T, D = rois[i]
            for ctr, nbr in pairs:
                for nb in rmax:
                    grids[i].build(X, T, nbr, nb * 0.01 * (1 + 1e-6))
                    for dmin in dsrf:
                        ps.spatstat(grids[i], D, ctr, dmin, (0.0, 0.01, nb), ks, check=False)

    plain_all()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plain_all()
    e1.record()
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    for gd in grids.values():
        gd.close()
    return {"workload": f"{len(rois)} ROIs, {n_ions} ions (log-uniform 1e4..1e7), k=1..20, r_max {{1,2,3}} nm, "
                        "d_srf {0,1,2} nm, pairs all-all/Sc-Sc/Al-Sc",
            "sweep_points": len(rois) * 27, "batched_ms": all_ms,
            "ion_queries_per_s": n_central_all / (all_ms * 1e-3),
            "subset_rois": len(sub), "subset_batched_ms": sub_ms, "subset_plain_ms": plain_ms,
            "plain_over_batched": plain_ms / sub_ms, "cell_scale": best_cs,
            "autotune_subset_ms": {f"cell_scale={k[0]}": round(v, 2) for k, v in sub_t.items()},
            "host_generation_s": gen_s,
            "timing": "CUDA events; batched = one CUDA-graph replay (grid builds + one persistent query "
                      "kernel + expansion); plain = one eager ps_spatstat per ROI and sweep point"}


def rank_reduce(dist, device, t_max, sums):
    """Whole-job numbers across ranks: the slowest rank's time and the summed counts.

    dist is torch.distributed (or None for one process); device is where the reduction
    tensors live (a CUDA device under NCCL, the CPU under gloo)."""
    import torch

    if dist is None:
        return float(t_max), [float(x) for x in sums]
    tt = torch.tensor([float(t_max)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    ss = torch.tensor([float(x) for x in sums], dtype=torch.float64, device=device)
    dist.all_reduce(ss)
    return float(tt.item()), [float(x) for x in ss.tolist()]


def run_gpu(args, wl_name, wl):
    import torch

    import paper_2004_05188_gb300 as ps

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    dev = torch.device("cuda", local)
    cloud = make_cloud(wl_name, seed_offset=1000 * rank)
    xyz, t, d = cloud
    N = xyz.shape[0]
    X = torch.from_numpy(xyz).to(dev)
    T = torch.from_numpy(t).to(dev)
    D = torch.from_numpy(d).to(dev)
    bins = wl["bins"]
    r_cut = float(np.float32(bins[0] + bins[1] * bins[2]))
    # kernel configuration per combination: measured by the autotuner on this cloud (untimed)
    tuned = {}
    for name, ctr, nbr in wl["combos"]:
        if args.no_autotune:
            tuned[name] = {"cell_scale": args.cell_scale, "dense_min": args.dense_min}
        else:
            from paper_2004_05188_gb300 import autotune

            tuned[name] = autotune.tune(X, T, D, nbr, ctr, wl["dsrf_min"], wl["bins"], wl["ks"])
    grids = [ps.Grid(N, tuned[name]["cell_scale"], tuned[name]["dense_min"]) for name, _, _ in wl["combos"]]
    nk = len(wl["ks"])
    outs = []
    for _ in wl["combos"]:
        outs.append(dict(rdf=torch.empty(bins[2], dtype=torch.int64, device=dev),
                         knn=torch.empty((nk, bins[2]), dtype=torch.int64, device=dev),
                         meta=torch.empty(ps.META_HEAD + 2 * nk, dtype=torch.int64, device=dev)))
    stream = torch.cuda.current_stream()
    # the type combinations are independent analyses: each runs on its own stream, so that the
    # short, latency-bound kernels of one overlap with the other's
    combo_streams = None
    if len(wl["combos"]) > 1 and not args.serial_combos:
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

    # correctness of the configuration before timing: device status words
    step()
    torch.cuda.synchronize()
    st = {"n_ions": N, "combos": []}
    n_queries = 0
    n_pairs = 0
    for (name, ctr, nbr), g, o in zip(wl["combos"], grids, outs):
        meta = o["meta"].cpu().numpy()
        if meta[3] != 0:
            raise RuntimeError(f"device status {meta[3]} for {name}")
        info = g.info()
        ctr_set = range(256) if ctr == "all" else ctr
        ntm = int(np.isin(t, list(ctr_set)).sum())
        stencil = 1 if tuned[name]["cell_scale"] >= 1.0 else 2
        st["combos"].append(dict(name=name, n_nbr=info["n_nbr"], n_cells=info["n_cells"], n_central=int(meta[0]),
                                 n_ctr_typed=ntm, n_pairs=int(meta[1]),
                                 candidates=candidate_tests(X, T, D, ctr, nbr, wl["dsrf_min"], info, stencil)))
        n_queries += int(meta[0])
        n_pairs += int(meta[1])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # dominant kernel family and its per-launch time: an eager pass with CUDA
    # events around every launch of the library (not the graph-timed region)
    fams = ["reset", "select", "geometry", "count", "scan", "scatter", "central", "query", "epilogue"]
    # (the combinations one after the other on one stream, so that every launch is timed alone)
    ps.prof_enable(fams)
    for _ in range(args.steps):
        flush.zero_()
        step(serial=True)
    torch.cuda.synchronize()
    prof = {f: ps.prof_read(f) for f in fams}
    ps.prof_enable([])
    shares = {f: v[1] for f, v in prof.items()}
    dom = max(shares, key=shares.get)
    dom_n, dom_ms = prof[dom]
    eager_ms = None

    # the timed step: the whole pass captured once in a CUDA graph, replayed per step
    graph = None
    kernels_per_step = None
    if not args.no_graph:
        lc = ps.launch_count()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        kernels_per_step = ps.launch_count() - lc
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()

    def timed_step():
        if graph is not None:
            graph.replay()
        else:
            step()

    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else
                           int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local]), args.clocks_csv)
    sampler.start()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    lc0 = ps.launch_count()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (not timed)
        ev0[k].record(stream)
        timed_step()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    launches = ps.launch_count() - lc0 if graph is None else kernels_per_step * args.steps
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    T_ms, (tot_q, tot_p) = rank_reduce(dist, dev, float(sum(step_ms)), [n_queries, n_pairs])
    value = tot_q * args.steps / (T_ms * 1e-3)

    # ---- e2e through the public API, inputs in pinned host memory ----
    e2e = None
    if not args.no_e2e:
        Xh = torch.from_numpy(xyz).pin_memory()
        Th = torch.from_numpy(t).pin_memory()
        Dh = torch.from_numpy(d).pin_memory()
        res_h = [{k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in o.items()} for o in outs]

        def d2h():
            for o, h in zip(outs, res_h):
                for k in o:
                    h[k].copy_(o[k], non_blocking=True)

        if graph is not None:
            # pipelined: every step copies its own inputs into one of two device buffer sets on a
            # copy stream, overlapping the previous step's compute; the compute stream replays
            # the graph captured for that buffer set and reads the results back.  No L2 flush:
            # the 137 MB of inputs per step exceed the 129 MB L2.
            XB, TB, DB = torch.empty_like(X), torch.empty_like(T), torch.empty_like(D)
            graph_b = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph_b):
                step(XB, TB, DB)
            sets, graphs = [(X, T, D), (XB, TB, DB)], [graph, graph_b]
            # the inputs are copied in n_cs contiguous slices on as many streams (several copy
            # engines share the host link)
            n_cs = args.copy_streams
            copy_ss = [torch.cuda.Stream(device=dev) for _ in range(n_cs)]
            ev_copy = [[torch.cuda.Event() for _ in range(n_cs)] for _ in range(2)]
            ev_used = [torch.cuda.Event(), torch.cuda.Event()]

            def slices(n):
                cut = [n * i // n_cs for i in range(n_cs + 1)]
                return [(cut[i], cut[i + 1]) for i in range(n_cs)]

            def run_e2e(n_steps):
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record(stream)
                for cs in copy_ss:
                    cs.wait_event(t0)
                for k in range(n_steps):
                    b = k % 2
                    for i, cs in enumerate(copy_ss):
                        with torch.cuda.stream(cs):
                            if k >= 2:
                                cs.wait_event(ev_used[b])
                            for dst, src in zip(sets[b], (Xh, Th, Dh)):
                                lo, hi = slices(src.shape[0])[i]
                                dst[lo:hi].copy_(src[lo:hi], non_blocking=True)
                            ev_copy[b][i].record(cs)
                    for i in range(n_cs):
                        stream.wait_event(ev_copy[b][i])
                    graphs[b].replay()
                    ev_used[b].record(stream)
                    d2h()
                t1.record(stream)
                torch.cuda.synchronize()
                return t0.elapsed_time(t1)

            run_e2e(4)
            E_local = run_e2e(args.steps)
            e2e_mode = (f"pipelined: H2D of step k+1 ({n_cs} copy streams) overlaps compute of step k "
                        "(two input buffer sets)")
        else:
            Xd, Td, Dd = torch.empty_like(X), torch.empty_like(T), torch.empty_like(D)

            def e2e_step():
                Xd.copy_(Xh, non_blocking=True)
                Td.copy_(Th, non_blocking=True)
                Dd.copy_(Dh, non_blocking=True)
                step(Xd, Td, Dd)
                d2h()

            for _ in range(2):
                e2e_step()
            torch.cuda.synchronize()
            e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
            for k in range(args.steps):
                flush.zero_()
                e0[k].record(stream)
                e2e_step()
                e1[k].record(stream)
            torch.cuda.synchronize()
            E_local = float(sum(a.elapsed_time(b) for a, b in zip(e0, e1)))
            e2e_mode = "serial: H2D, compute, D2H per step, L2 flushed between steps"
        E_ms, _ = rank_reduce(dist, dev, E_local, [])
        h2d = xyz.nbytes + t.nbytes + d.nbytes
        d2h_bytes = sum(v.numel() * v.element_size() for o in outs for v in o.values())
        e2e = {"value": tot_q * args.steps / (E_ms * 1e-3), "unit": "ion-queries/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h_bytes, "ms_per_step": E_ms / args.steps, "mode": e2e_mode}

    # ---- roofline of the dominant kernel family ----
    peak, peak_kind = load_peaks()
    alg = algorithmic_bytes(dom, st)
    launches_per_step = max(1, dom_n // max(1, args.steps))
    per_launch_bytes = alg / launches_per_step
    avg_ms = dom_ms / max(1, dom_n)
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9 if avg_ms > 0 else 0.0
    kcfg = {name: {"cell_scale": float(tuned[name]["cell_scale"]), "dense_min": int(tuned[name]["dense_min"])}
            for name, _, _ in wl["combos"]}
    common = {"kernel": dom, "peak_source": peak_kind, "avg_launch_us": avg_ms * 1e3, "launches": dom_n,
              "timing": "CUDA events around each launch, eager pass of the step with the combinations one after the other",
              "time_share": shares[dom] / max(1e-12, sum(shares.values())),
              "shares": {k: round(v / max(1e-12, sum(shares.values())), 4) for k, v in shares.items()}}
    hbm = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "algorithmic_bytes_per_launch": per_launch_bytes}
    if dom == "query":
        # the pair test is the work: FP32 arithmetic on L2-resident records (DRAM traffic is a few MB)
        cands = sum(c["candidates"] for c in st["combos"])
        flops = FLOPS_PER_CANDIDATE * cands / launches_per_step
        alu_peak, mhz = alu_peak_tflops()
        alu = flops / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else 0.0
        roofline = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu / alu_peak,
                    "traffic": stored_traffic(wl_name, kcfg), "traffic_unit": "DRAM bytes per launch (ncu)",
                    "flops_per_launch": flops, "candidate_tests_per_step": cands,
                    "peak_derivation": f"{N_SM} SMs x {FP32_LANES} FP32 lanes x {mhz:.0f} MHz, 1 op/lane/clock",
                    "hbm": hbm, **common}
    else:
        roofline = {"bound": "hbm", **{k: v for k, v in hbm.items() if k != "algorithmic_bytes_per_launch"},
                    "traffic": None, **common}

    forms = None
    if rank == 0 and not args.no_forms:
        forms = {"soft": measure_soft(args, dev)}
        if args.batch_rois > 0:
            forms["batched"] = measure_batched(args, dev)
        forms["sdm"] = measure_sdm(args, dev)
        forms["cluster"] = measure_cluster(args, dev)

    # ---- cpu baseline: the oracle on a bounded sample (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import concurrent.futures as cf

        # all host cores: independent oracle runs over consecutive z-slabs of centrals (exact sum)
        cores = host_cores()
        with cf.ThreadPoolExecutor(max_workers=cores) as pool:
            orc, parts, frac, nq, _ = oracle_sample_parallel(wl, cloud, pool, cores, target_s=2.0)
            reps = 0
            t0 = time.perf_counter()
            while reps < 3 or time.perf_counter() - t0 < 10.0:
                oracle_step_parts(orc, parts, wl, pool)
                reps += 1
                if time.perf_counter() - t0 > 30.0:
                    break
            dt = time.perf_counter() - t0
        # and one core, for reference
        orc, samp, frac1, nq1, _ = oracle_sample(wl_name, wl, cloud, target_s=1.0)
        t1 = time.perf_counter()
        reps1 = 0
        while reps1 < 2 or time.perf_counter() - t1 < 3.0:
            oracle_step(orc, samp, wl)
            reps1 += 1
        dt1 = time.perf_counter() - t1
        cpu = {"value": nq * reps / dt, "unit": "ion-queries/s", "cores": cores, "kind": "oracle",
               "sample": f"z-slab with {frac:.3f} of the height split in {cores} slabs of centrals (+2 nm halo "
                         f"each), one host thread each; {nq} centrals, {reps} runs",
               "value_1core": nq1 * reps1 / dt1}

    if rank == 0:
        line = {
            "metric": "ion-queries/s (exact kNN+RDF)", "value": value, "unit": "ion-queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": T_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl["desc"], "n_ions": N, "centrals_per_step": n_queries,
                       "kernel_config": {k: {"cell_scale": v["cell_scale"], "dense_min": v["dense_min"]}
                                         for k, v in tuned.items()},
                       "autotune": {k: v.get("timings_ms") for k, v in tuned.items()},
                       "neighbour_pairs_per_step": n_pairs, "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"replicas x{world} (independent specimens, no collective)",
                       "combo_streams": len(combo_streams) if combo_streams else 1},
            "neighbour_pairs_per_s": tot_p * args.steps / (T_ms * 1e-3),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps, "clocks": clocks, "wall_s_timed_loop": wall,
            "cuda_graph": graph is not None, "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    for g in grids:
        g.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="needle8m", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--clocks-csv", default=None, help="file for the raw nvidia-smi clock samples of the timed region "
                                                         "(default: a temporary file)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--copy-streams", type=int, default=1, help="streams for the e2e input copies (one is fastest)")
    ap.add_argument("--serial-combos", action="store_true", help="run the type combinations one after the other "
                    "on one stream (default: one stream each)")
    ap.add_argument("--no-graph", action="store_true", help="launch the step eagerly instead of replaying a CUDA graph")
    ap.add_argument("--no-forms", action="store_true", help="skip the smoothed-RDF and batched measurements")
    ap.add_argument("--batch-rois", type=int, default=256, help="ROIs of the batched measurement (0 skips it)")
    ap.add_argument("--batch-cell-scale", type=float, default=1.0)
    ap.add_argument("--cell-scale", type=float, default=1.0, help="cell edge / r_cut (>= 0.5)")
    ap.add_argument("--dense-min", type=int, default=0, help="centrals per cell for the staged CTA kernel (0: never)")
    ap.add_argument("--no-autotune", action="store_true", help="use --cell-scale/--dense-min instead of the autotuner")
    ap.add_argument("--only-form", choices=["soft", "batched", "sdm", "cluster"],
                    help="measure only this form (no exact step line)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    wl = dict(WORKLOADS[args.workload])
    r0, dr, stop = wl["spec"]
    wl["bins"] = (r0, dr, int(round((stop - r0) / dr)))
    if args.impl == "reference":
        return run_reference(args, args.workload, wl)
    import __graft_entry__

    __graft_entry__.build()
    if args.only_form:
        import torch

        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        torch.cuda.set_device(dev)
        fn = {"soft": measure_soft, "batched": measure_batched, "sdm": measure_sdm,
              "cluster": measure_cluster}[args.only_form]
        print(json.dumps({"form": args.only_form, **fn(args, dev)}), flush=True)
        return 0
    return run_gpu(args, args.workload, wl)


if __name__ == "__main__":
    sys.exit(main())
