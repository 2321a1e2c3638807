"""Replicas-only multi-GPU logic of bench.py on CPU with gloo, world size 2:
every rank solves its own instance, the job time is the max over ranks and
the value counts the DOFs of all ranks."""
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
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = 1.5 if rank == 0 else 2.5  # seconds of this rank's timed steps
    value, t = bench.aggregate(local, 1000, 4, dist)
    q.put((rank, value, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_aggregate_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t in res:
        assert t == pytest.approx(2.5)
        assert value == pytest.approx(1000 * 4 * 2 / 2.5 / 1e6)


def test_single_process_aggregate():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    value, t = bench.aggregate(2.0, 823875, 5, None)
    assert t == 2.0 and value == pytest.approx(823875 * 5 / 2.0 / 1e6)
