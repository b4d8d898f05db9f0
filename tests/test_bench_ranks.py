"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

The solver does not shard: N GPUs run N replicas, the step time is the
maximum over ranks and the value counts the lattice updates of all ranks.
Here two gloo processes stand in for the ranks and exercise that host logic.
"""
import json
import multiprocessing as mp
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


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]                      # rank 1 is the slower replica
    got = bench.max_over_ranks(ms, "cpu", world)
    val = bench.whole_job_mlups(world, 1000, 10, got * 1e-3)
    dist.destroy_process_group()
    q.put((rank, got, val))


def test_max_over_ranks_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, val in out:
        assert got == 20.0                        # both ranks see the slowest time
        assert val == pytest.approx(2 * 1000 * 10 / 0.020 / 1e6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, "cpu", 1) == 3.25
    assert bench.whole_job_mlups(1, 8, 5, 2.0) == 8 * 5 / 2.0 / 1e6


def test_reference_arm_prints_on_rank_zero_only():
    # the reference arm under torchrun: rank 0 prints one JSON line, the
    # other ranks exit 0 without work
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1


def test_equilibrium_workloads_keep_their_step_count(monkeypatch):
    # the angle and W-sweep workloads run to equilibrium: the timed-step
    # default of the throughput workloads must not shorten them
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(steps=2000)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "angles3d"])
    assert bench.long_solve_steps(args) == 20000
    for given in (["--steps", "2000"], ["--steps=2000"]):
        monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "angles3d"] + given)
        assert bench.long_solve_steps(args) == 2000
