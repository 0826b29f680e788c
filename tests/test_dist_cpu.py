"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The codec shards with no data-path collective (chunks and tensors are
independent, ZipNN Sec. 5.1); the only collectives are the timing barrier and
the max-over-ranks reduction, tested here without a GPU."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, loc = bench.dist_info()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    got = bench.all_max([float(rank + 1), 10.0 - rank], world)
    dist.destroy_process_group()
    q.put((rank, (w, r, loc), got))


def test_max_over_ranks_and_barrier_gloo():
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
    for rank, info, got in res:
        assert info == (2, rank, rank)
        assert got == [2.0, 10.0]
