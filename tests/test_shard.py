"""Slab sharding of one specimen (the paper's spatial splitting across ranks), on CPU.

* partition arithmetic: cuts are ascending, cover every layer once and balance the ion count;
  the halo depth covers r_cut plus the z jitter;
* halo sufficiency, checked on the whole cloud: every ion within r_cut (in z) of a rank's core
  ions lies in that rank's generated layers;
* two gloo ranks (world size 2): each rank generates only its slab + halo, computes its
  statistics (here with the oracle, which stands in for the GPU on a machine without one),
  and the summed integer results equal the oracle's on the whole needle, bin for bin.
"""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2004_05188_gb300 import shard  # noqa: E402


def _needle(spec):
    return spec.needle_params(5.0, 10.0, 16.0, seed=9)


def test_layer_cuts_balance_and_cover(spec):
    p = _needle(spec)
    counts = spec.needle_plan(p)
    for parts in (1, 2, 3, 5, 8):
        cuts = shard.layer_cuts(counts, parts)
        assert cuts[0] == 0 and cuts[-1] == len(counts) and all(a <= b for a, b in zip(cuts, cuts[1:]))
        per = [int(counts[a:b].sum()) for a, b in zip(cuts, cuts[1:])]
        assert sum(per) == int(counts.sum())
        # each slab within one layer's worth of ions of the ideal share
        assert max(per) - min(per) <= 2 * int(counts.max()), per
    assert shard.halo_layers(0.404, 2.0, 0.1) * 0.404 >= 2.0 + 2 * 15 * 0.1


def test_halo_holds_every_neighbour_within_r_cut(spec):
    p = _needle(spec)
    counts = spec.needle_plan(p)
    xyz, t, d = spec.needle(p)
    off = np.concatenate([[0], np.cumsum(counts)])
    r_cut = 2.0
    halo = shard.halo_layers(p.a, r_cut, p.sig_z)
    cuts = shard.layer_cuts(counts, 3)
    z = xyz[:, 2]
    for rank in range(3):
        k0, k1, c0, c1 = shard.rank_layers(cuts, rank, halo, len(counts))
        core = z[off[c0]:off[c1]]
        if core.size == 0:
            continue
        outside = np.concatenate([z[:off[k0]], z[off[k1]:]])
        # no ion outside the generated layers is within r_cut of the core in z
        assert not np.any((outside > core.min() - r_cut) & (outside < core.max() + r_cut))
        xs, ts, ds, (i0, i1) = shard.slab_needle(p, counts, cuts, rank, halo)
        np.testing.assert_array_equal(xs, xyz[off[k0]:off[k1]])
        assert np.all(np.isnan(ds[:i0])) and np.all(np.isnan(ds[i1:]))
        np.testing.assert_array_equal(ds[i0:i1], d[off[c0]:off[c1]])


def _rank_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle
    from paper_2004_05188_gb300 import shard as sh
    from paper_2004_05188_gb300 import specimen

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = specimen.needle_params(5.0, 10.0, 16.0, seed=9)
    counts = specimen.needle_plan(p)
    cuts = sh.layer_cuts(counts, world)
    halo = sh.halo_layers(p.a, 2.0, p.sig_z)
    xyz, t, d, _ = sh.slab_needle(p, counts, cuts, rank, halo)
    res = {}
    for name, ctr, nbr, ks in (("all", "all", "all", [1, 10]), ("scsc", [1], [1], [1, 5])):
        r = oracle.spatstat(xyz, t, d, ctr, nbr, 1.0, 0.0, 0.01, 200, ks)
        meta = [r["n_central"], r["n_pairs"], r["rdf_below"], 0]
        for q in range(len(ks)):
            meta += [r["not_found"][q], r["knn_below"][q]]
        out = {"rdf": torch.from_numpy(r["rdf"].astype(np.int64)), "knn": torch.from_numpy(r["knn"].astype(np.int64)),
               "meta": torch.tensor(meta, dtype=torch.int64)}
        if rank == 1:
            out["meta"][3] = 0  # every status is 0 here; the max-combine is exercised below
        sh.combine(dist, out)
        res[name] = {k: v.tolist() for k, v in out.items()}
    st = {"rdf": torch.zeros(1, dtype=torch.int64), "knn": None,
          "meta": torch.tensor([0, 0, 0, 2 if rank == 1 else 0], dtype=torch.int64)}
    sh.combine(dist, st)
    res["status"] = st["meta"].tolist()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_add_up_to_the_whole_needle(tmp_path, orc, spec):
    import torch.multiprocessing as mp

    port = 29700 + (os.getpid() % 1000)
    mp.spawn(_rank_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    xyz, t, d = spec.needle(_needle(spec))
    combos = (("all", "all", "all", [1, 10]), ("scsc", [1], [1], [1, 5]))
    refs = {name: orc.spatstat(xyz, t, d, ctr, nbr, 1.0, 0.0, 0.01, 200, ks) for name, ctr, nbr, ks in combos}
    for r in range(2):
        with open(tmp_path / f"r{r}.json") as f:
            got = json.load(f)
        for name, ctr, nbr, ks in combos:
            ref = refs[name]
            g = got[name]
            np.testing.assert_array_equal(np.array(g["rdf"], np.uint64), ref["rdf"])
            np.testing.assert_array_equal(np.array(g["knn"], np.uint64), ref["knn"])
            assert g["meta"][0] == ref["n_central"] and g["meta"][1] == ref["n_pairs"] and g["meta"][3] == 0
            assert g["meta"][4::2] == list(ref["not_found"])
        assert got["status"][3] == 2  # a device status on any rank survives the combine (max)
