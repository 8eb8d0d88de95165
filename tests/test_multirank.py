"""Host logic of the N > 1 bench path (replicas, no data-path collective) on
CPU ranks over gloo: the job time is the slowest rank's, the job value counts
every rank's simulated time, and the reference arm does its work on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 37.0 * rank          # rank 1 is the slow one
    got = bench.max_over_ranks(ms, world, "cpu")
    val = bench.job_value(got, 5, world)
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": got, "value": val}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo_world2(tmp_path):
    port = 29500 + (os.getpid() % 2000)
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    assert r[0]["max"] == r[1]["max"] == 137.0
    import bench
    # 5 steps of 0.1 time units on each of 2 replicas = 1.0 unit of simulated time in 137 ms
    assert abs(r[0]["value"] - 0.137 / (bench.SIM_TIME_PER_STEP * 5 * 2)) < 1e-15
    assert bench.job_value(137.0, 5, 1) == pytest.approx(2 * r[0]["value"])


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0
    assert p.stdout.strip() == ""
