"""The multi-process (replica) accounting of bench.py on CPU: world size 2, gloo backend.

Each rank times its own solve; the job's time is the slowest rank's and its work the sum.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1712_01505_gb300.replicas import replica_reduce

    ms, units = replica_reduce(10.0 + 5.0 * rank, 100.0 * (rank + 1), dist, torch.device("cpu"))
    out[rank] = (ms, units)
    dist.destroy_process_group()


def test_replica_reduce_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (15.0, 300.0)


def test_replica_reduce_single_process_is_identity():
    from paper_1712_01505_gb300.replicas import replica_reduce

    assert replica_reduce(3.5, 7.0) == (3.5, 7.0)
