"""The N > 1 path of bench.py on CPU: two gloo ranks, each reporting its own
timed total and units, aggregated as max time and summed units (replicas,
no collective on the data path)."""

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


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate(10.0 + rank, 1000 * (rank + 1), world)
    q.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in (0, 1)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for _, t, u in got:
        assert t == 11.0      # max over ranks of the timed totals
        assert u == 3000.0    # units of all ranks


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate(5.5, 42, 1) == (5.5, 42.0)
