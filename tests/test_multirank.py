"""The multi-rank host path of bench.py on CPU: two gloo ranks.

For N > 1 the bench runs one independent replica of the step per GPU; the
only cross-rank steps are the barrier and the maximum of the timed regions
over ranks, from which the whole-job rate is formed.  Those steps are
checked here with the gloo backend, and the reference arm's rule that only
rank 0 runs and prints.
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r times (10 (r+1)) ms for the device region and (50 - r) s end to end
        ms_max, e2e_max = bench.max_over_ranks([10.0 * (rank + 1), 50.0 - rank])
        value = bench.replica_throughput(1.0e6, ms_max / 1e3, dist.get_world_size())
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"ms_max": ms_max, "e2e_max": e2e_max, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for g in got:
        # the slowest rank's time on every rank, element by element
        assert g["ms_max"] == 20.0
        assert g["e2e_max"] == 50.0
        # 2 replicas x 1e6 units in 20 ms
        assert g["value"] == pytest.approx(1.0e8, rel=1e-15)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([3.0, 1.5]) == [3.0, 1.5]
    assert bench.replica_throughput(5.0, 0.5, 1) == 10.0
    with pytest.raises(ValueError):
        bench.replica_throughput(5.0, 0.0, 2)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "2", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
