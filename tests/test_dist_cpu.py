"""The bench's multi-rank plumbing on CPU: two gloo ranks, barrier, max-over-ranks time and the
sum of the units both processed (the path is run as replicas: no data-path collective)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    d.barrier()
    t = d.max(10.0 + rank)                   # each rank's own elapsed time
    n = d.sum(1000.0 * (rank + 1))           # units each rank rendered
    d.barrier()
    q.put((rank, t, n, d.world))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_units():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 11.0, 3000.0, 2), (1, 11.0, 3000.0, 2)]
