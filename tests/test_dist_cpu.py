"""The multi-rank harness of bench.py on CPU: world size 2 over gloo.

bench.py runs one independent replica per GPU (no data-path collective: the
path shards over (atom, energy) units, but one structure's sigma is a single
sum and the workload fits one GPU); the only cross-rank operations are the
barrier around the timed region and the max over ranks of the step time.
"""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys
sys.path.insert(0, %(root)r)
import bench
rank, world, local = bench.dist_env()
active = bench.init_dist(world, "gloo")
assert active and world == 2
bench.barrier(active)
m = bench.max_over_ranks(10.0 * (rank + 1), active)
assert m == 20.0, m
# the reference arm: rank 0 alone prints; other ranks return 0 without work
if rank != 0:
    class A: gpus = 2; steps = 1; warmup = 0
    assert bench.run_reference(A()) == 0
print("rank", rank, "ok", m, flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_barrier_and_max_over_ranks():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER % {"root": ROOT}], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
    outs = []
    for p in procs:
        out, _ = p.communicate(timeout=120)
        outs.append(out)
        assert p.returncode == 0, out
    assert "rank 0 ok 20.0" in outs[0] and "rank 1 ok 20.0" in outs[1]


def test_replica_value_is_whole_job():
    """value = world * units / max step time (weak scaling over replicas)."""
    units, world, ms = 512, 4, 100.0
    assert abs(world * units / (ms * 1e-3) - 20480.0) < 1e-9
