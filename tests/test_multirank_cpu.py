"""The N > 1 host path of bench.py on CPU: two gloo ranks, the barrier and
the max-over-ranks reduction used for whole-job timing (replicas only: no
collective touches the data path)."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
rank, world, local = bench.dist_init()
bench.barrier(world)
t = bench.max_over_ranks(1.5 + rank, world)
bench.barrier(world)
print(json.dumps({{"rank": rank, "world": world, "max": t}}))
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_rank_barrier_and_max():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    import json
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    assert sorted(r["rank"] for r in res) == [0, 1]
    assert all(r["world"] == 2 and r["max"] == 2.5 for r in res)


def test_reference_arm_under_two_ranks_prints_once():
    """Under a two-rank launch the reference arm runs on rank 0 only: one JSON
    line in all, both ranks exit 0."""
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "bench.py", "--impl", "reference", "--workload", "disk",
                                       "--gpus", "2", "--steps", "1", "--warmup", "1"], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    lines = [ln for o, _ in outs for ln in o.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    import json
    assert json.loads(lines[0])["impl"] == "reference"
    assert not outs[1][0].strip()
