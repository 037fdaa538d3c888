"""The N > 1 harness of bench.py (replicas, no data-path collective) on CPU
with the gloo backend, world size 2: the step time reported is the max over
ranks, and each replica draws its own seed."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
    res = (bench.allreduce_max(ms, world), bench.replica_seed(rank))
    with open(os.path.join(outdir, f"{rank}.txt"), "w") as f:
        f.write(f"{res[0]} {res[1]}")
    bench.barrier(world)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replica_harness_world_size_2(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    out = [open(tmp_path / f"{r}.txt").read().split() for r in range(world)]
    assert float(out[0][0]) == float(out[1][0]) == 15.0
    assert out[0][1] != out[1][1]
