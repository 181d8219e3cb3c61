"""The benchmark's multi-rank logic on CPU ranks (gloo, world size 2): max-over-ranks time, summed
counts, and the reference arm doing no work on ranks other than 0."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, sums = bench.rank_reduce(dist, "cpu", 10.0 + rank, [100 * (rank + 1), 7])
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"t": t, "sums": sums}, f)
    dist.destroy_process_group()


def test_rank_reduce_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = 29500 + (os.getpid() % 1000)
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        with open(tmp_path / f"r{r}.json") as f:
            d = json.load(f)
        assert d["t"] == 11.0
        assert d["sums"] == [300.0, 14.0]


def test_rank_reduce_single_process():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.rank_reduce(None, "cpu", 3.5, [1, 2]) == (3.5, [1.0, 2.0])


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
