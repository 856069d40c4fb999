"""The multi-GPU form of the benchmark is replicas: each rank renders its own poses with no
data-path collective, the job time is the max over ranks and the value the whole job's
throughput.  This checks that host logic with two gloo ranks on the CPU (127.0.0.1), and
that the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    poses = bench.rank_poses(rank, 100, 8)
    ms = bench.max_over_ranks(1.0 + 0.5 * rank, dist, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, poses)
    res = {"rank": rank, "poses": gathered, "ms": ms,
           "value": bench.job_throughput(world, 10, 307200, ms)}
    dist.barrier()
    dist.destroy_process_group()
    with open(out % rank, "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    out = str(tmp_path / "rank%d.json")
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn")
    res = [json.load(open(out % r)) for r in range(world)]
    for r in res:
        assert r["ms"] == 1.5                      # the slowest rank's time on every rank
        assert abs(r["value"] - 2 * 10 * 307200 / 1.5e-3 / 1e6) < 1e-9
        p0, p1 = r["poses"]
        assert len(p0) == len(p1) == 8 and not set(p0) & set(p1)   # different poses per rank
    assert res[0]["poses"] == res[1]["poses"]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.rank_poses(0, 5, 7) == [0, 1, 2, 3, 4, 0, 1]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
