"""The sharded transform's host logic (paper_1001_5272_gb300/shard.py) on
CPU: the partition, the exchanges and the step order, with the device steps
replaced by oracle-built stand-ins (tests/shard_cpu_ops.py).  The assembled
result must equal the oracle's Algorithm 1 on the whole vector, and the
sharded inverse must return the input, for every number of parts; two gloo
ranks run the distributed driver (point-to-point exchanges)."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from oracle import field as F  # noqa: E402
from oracle import native as NV  # noqa: E402
from paper_1001_5272_gb300 import shard  # noqa: E402
from paper_1001_5272_gb300 import tft  # noqa: E402

from shard_cpu_ops import CpuOps  # noqa: E402


def _x(pid, n, seed):
    p = F.PRIME_BY_ID[pid].p
    x = np.random.default_rng(seed).integers(0, p, n, dtype=np.uint64)
    return torch.from_numpy(x.view(np.int64).copy())


def _layout(pid, n, parts):
    return shard.Layout.for_plan(tft.tft_describe_plan(pid, n), n, parts)


def test_layout_round_trips():
    L = _layout(2, 70001, 4)
    assert (L.R, L.W, L.a, L.b) == (512, 128, 136, 369)
    assert [L.long_cols(p) for p in range(4)] == [128, 128, 113, 0]
    assert [L.rows_of(p) for p in range(4)] == [(0, 34), (34, 68),
                                                (68, 102), (102, 136)]
    x = _x(2, 70001, 1)
    assert torch.equal(L.vector_of_blocks([L.block_of(x, p)
                                           for p in range(4)]), x)
    assert torch.equal(L.vector_of_rows([L.rows_piece(x, p)
                                         for p in range(4)],
                                        L.last_piece(x)), x)
    with pytest.raises(ValueError):
        shard.Layout(70001, 9, 136, 369, 3)


@pytest.mark.parametrize("pid,n", [(2, 70001), (2, 70144), (1, 100003)])
@pytest.mark.parametrize("parts", [1, 2, 4, 8])
def test_sharded_forward_and_inverse_in_one_process(pid, n, parts):
    L = _layout(pid, n, parts)
    ops = CpuOps(pid, L)
    x = _x(pid, n, n + parts)
    rows, last = shard.forward_local(L, ops, [L.block_of(x, p)
                                              for p in range(parts)])
    X = L.vector_of_rows(rows, last)
    ref = NV.alg1_tft(pid, x.numpy().view(np.uint64))
    assert np.array_equal(X.numpy().view(np.uint64), ref)
    blocks = shard.inverse_local(L, ops, [L.rows_piece(X, p)
                                          for p in range(parts)],
                                 L.last_piece(X) if L.b else None)
    assert torch.equal(L.vector_of_blocks(blocks), x)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, pid, n, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch.distributed as dist
    from shard_cpu_ops import CpuOps as Ops
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L = _layout(pid, n, world)
    ops = Ops(pid, L)
    comm = shard.DistComm()
    x = _x(pid, n, 7)
    rows, last = shard.forward_rank(L, ops, comm, L.block_of(x, rank))
    q.put(("fwd", rank, rows.numpy().copy(),
           None if last is None else last.numpy().copy()))
    block = shard.inverse_rank(L, ops, comm, rows.clone(),
                               None if last is None else last.clone())
    q.put(("inv", rank, block.numpy().copy(), None))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_transform_on_gloo_ranks(world):
    pid, n = 2, 70001
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, pid, n, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(2 * world)]
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    L = _layout(pid, n, world)
    fwd = {r: (a, b) for k, r, a, b in got if k == "fwd"}
    inv = {r: a for k, r, a, _ in got if k == "inv"}
    X = L.vector_of_rows([torch.from_numpy(fwd[r][0]) for r in range(world)],
                         torch.from_numpy(fwd[world - 1][1]))
    x = _x(pid, n, 7)
    assert np.array_equal(X.numpy().view(np.uint64),
                          NV.alg1_tft(pid, x.numpy().view(np.uint64)))
    back = L.vector_of_blocks([torch.from_numpy(inv[r])
                               for r in range(world)])
    assert torch.equal(back, x)
