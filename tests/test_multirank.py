"""bench.py's multi-rank host logic on CPU with gloo, world size 2: every
rank solves its own copy of the batch (no collective on the data path); the
step time reported is the max over ranks, and the whole-job rate counts the
queries of all ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1000.0, 1500.0][rank]
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    qs = bench.job_rate(64, ms, world)
    out[rank] = (ms, qs)
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest():
    port = free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1]
    ms, qs = out[0]
    assert ms == 1500.0
    assert abs(qs - 2 * 64 / 1.5) < 1e-9
