"""The N > 1 host logic of bench.py on CPU: two gloo ranks run replicas and
the whole-job value is the work of all ranks over the slowest rank's time
(no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    t, w = bench.aggregate(100.0 + 50.0 * rank, 1000.0 * (rank + 1))
    q.put((rank, t, w))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, w in res:
        assert t == 150.0  # max over ranks
        assert w == 3000.0  # sum of the work of both replicas


def test_single_process_aggregate():
    import bench
    assert bench.aggregate(12.5, 7.0) == (12.5, 7.0)
