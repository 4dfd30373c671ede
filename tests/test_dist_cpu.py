"""The multi-rank plumbing of bench.py on CPU (gloo, world size 2).

The solver does not shard: `bench.py --gpus N` runs N independent replicas, one per
rank, and reports the summed unknowns over the slowest rank's time.  These tests cover
that host logic without a GPU: the barrier, the max over ranks, the replica
accounting, and the reference arm running on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["PD_ROOT"])
import torch
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import bench
rank, world, local = bench.dist_env()
bench.barrier(world)
m = bench.max_over_ranks(1.5 + rank, world, torch.device("cpu"))
v = bench.replica_throughput(1000, 4, world, m)
print(json.dumps({"rank": rank, "world": world, "local": local, "max": m, "value": v}))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_barrier_max_and_replica_accounting_with_gloo():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE="2",
                   LOCAL_RANK=str(r), PD_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["world"] == 2 and o["local"] == o["rank"]
        assert o["max"] == 2.5  # the slowest rank's time on every rank
        # 1000 unknowns x 4 steps on each of 2 replicas in 2.5 ms
        assert o["value"] == pytest.approx(1000 * 4 * 2 / 2.5e-3)


def test_reference_arm_runs_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
