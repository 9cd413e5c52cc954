"""The multi-replica timing of bench.py over a world of 2 CPU ranks (gloo): the slowest rank's
time and the units of all ranks make the whole-job throughput."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 if rank == 0 else 250.0           # rank 1 is slower
    units = 1000 * (rank + 1)                    # ranks process different amounts
    t, value = bench.aggregate_replicas(ms, units, steps=10)
    out.put((rank, t, value))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, t, value in res:
        assert t == 250.0                                   # max over ranks
        assert value == pytest.approx(3000 * 10 / 0.25)     # all ranks' units / slowest time
