"""Host logic of bench.py's N > 1 path, on CPU: two gloo ranks (world size 2).

The GPU arm runs one independent replica per rank; the job time is the max over ranks and the
job rate counts every replica's cells.  The reference arm runs on rank 0 only.
"""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, secs, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.replica_max(secs[rank], dist, "cpu")
        out[rank] = (t, bench.job_rate(world, 512 * 512, 10, t))
    finally:
        dist.destroy_process_group()


def test_replica_time_is_the_max_over_ranks_and_rate_counts_all_replicas():
    world, port = 2, _free_port()
    secs = [0.25, 0.5]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, secs, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == 0.5
        assert rate == pytest.approx(2 * 512 * 512 * 10 / 0.5)


def test_single_process_needs_no_collective():
    import bench
    assert bench.replica_max(0.3, None, "cpu") == 0.3
    assert bench.job_rate(1, 100, 4, 2.0) == 200.0


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
