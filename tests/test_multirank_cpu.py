"""World-size-2 gloo test (CPU) of the benchmark's multi-rank host logic:
independent replicas, whole-job value = all ranks' events / slowest rank's
time; only rank 0 prints."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    events = 1000.0 * (rank + 1)
    seconds = 2.0 + rank
    v, t, ev = bench.aggregate(world, rank, events, seconds)
    q.put((rank, v, t, ev))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, t, ev in res:
        assert t == 3.0            # slowest rank
        assert ev == 3000.0        # all ranks' events
        assert abs(v - 1000.0) < 1e-12
