"""Sharded decoding of one checkpoint, host side (CPU only; gloo ranks).

The chunks of a set of containers are split into one contiguous range per rank
by zipnn_partition_chunks (host code of the C-ABI library, no CUDA call), from
the containers' maps (ZipNN Sec. 5.1: chunks are independent and the map locates
every chunk and byte group).  Checked here: every chunk is owned by exactly one
rank, the decode traffic (stored payload bytes + original bytes per chunk,
recomputed from the maps in Python) is balanced within 5%, and the bytes each
rank decodes for its range, gathered over gloo with world sizes 2 and 3,
reassemble into exactly the single-rank decode.  On these CPU ranks the
per-rank decode is the oracle's (a whole-container decode cut to the rank's
extents); the GPU range plans are tested in test_shard_gpu.py."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle as O
from paper_2411_05239_gb300 import workloads as W
from paper_2411_05239_gb300 import zipnn as Z
from tests import spec_decoder

CHUNK = 16384


def _inputs():
    rng = np.random.default_rng(5)
    xs = [
        (O.BF16, W.gaussian(1_000_003, 0.02, 1).view(torch.int16).numpy(), None),
        (O.BF16, np.full(4096, 0x3F80, dtype=np.uint16), None),            # a norm vector
        (O.FP32, W.gaussian(300_001, 0.05, 2, torch.float32).numpy(), None),
        (O.U8, rng.integers(0, 7, size=200_011).astype(np.uint8), None),
        (O.BF16, np.zeros(0, dtype=np.uint16), None),                      # empty tensor
        (O.FP16, W.gaussian(500_000, 0.02, 3, torch.float16).view(torch.int16).numpy(), None),
    ]
    nxt, base = W.delta_pair(400_000, seed=4)
    xs.append((O.BF16, nxt.view(torch.int16).numpy(), base.view(torch.int16).numpy()))
    return xs


def _containers():
    out = []
    for dt, x, b in _inputs():
        s = O.compress(x, dt, CHUNK) if b is None else O.delta(x, b, dt, CHUNK)
        out.append((s, x, b))
    return out


def _zs(stream: bytes) -> Z.ZStream:
    h = spec_decoder.parse(stream)
    zs = Z.ZStream()
    zs.nbytes = len(stream)
    zs.orig_nbytes = h["nbytes"]
    zs.dtype = h["dtype"]
    zs.flags = h["flags"]
    zs.chunk_bytes = h["chunk_bytes"]
    zs.lanes = h["lanes"]
    zs.n_chunks = h["chunks"]
    zs.n_groups = h["groups"]
    return zs


def _weights(stream: bytes) -> list[int]:
    """Decode traffic per chunk, from the map (independent of the library)."""
    p = spec_decoder.parse(stream)
    G, C, n = p["groups"], p["chunk_bytes"], p["chunks"]
    out = []
    for c in range(n):
        w = min(C, p["nbytes"] - c * C)
        for g in range(G):
            off, size, mode, value = p["entries"][c * G + g][:4]
            if mode in (O.RAW, O.HUFF, 4):                 # 4: SPARSE
                w += (size + 15) // 16 * 16
        out.append(w)
    return out


def test_partition_owns_every_chunk_once_and_balances():
    conts = _containers()
    zss = [_zs(s) for s, _, _ in conts]
    w = [v for s, _, _ in conts for v in _weights(s)]
    total = sum(w)
    for world in (1, 2, 3, 4, 7):
        b = Z.partition_chunks(zss, [s for s, _, _ in conts], world)
        assert len(b) == world + 1 and b[0] == 0 and b[-1] == len(w)
        assert all(b[r] <= b[r + 1] for r in range(world))
        owned = [r for r in range(world) for _ in range(b[r], b[r + 1])]
        assert len(owned) == len(w)                       # every chunk exactly once
        share = [sum(w[b[r]:b[r + 1]]) for r in range(world)]
        assert sum(share) == total
        assert max(share) <= total / world + max(w)       # within one chunk of equal
        assert max(share) <= 1.05 * total / world         # and within 5% here


def test_partition_rejects_bad_arguments():
    conts = _containers()
    zss = [_zs(s) for s, _, _ in conts]
    with pytest.raises(Z.ZipnnError):
        Z.partition_chunks(zss, [s for s, _, _ in conts], 0)
    bad = bytearray(conts[0][0])
    bad[64 + 12] = 9                                     # unknown mode in the first entry
    with pytest.raises(Z.ZipnnError) as e:
        Z.partition_chunks(zss[:1], [bytes(bad)], 2)
    assert e.value.status == -3


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    conts = _containers()
    zss = [_zs(s) for s, _, _ in conts]
    b = Z.partition_chunks(zss, [s for s, _, _ in conts], world)
    # this rank decodes only its range: per container, the extent of its chunks
    mine = []
    for i, ext in enumerate(Z.range_extents(zss, b[rank], b[rank + 1])):
        if ext is None:
            continue
        _, start, size = ext
        s, x, base = conts[i]
        y = O.decompress(s, base)
        mine.append((i, start, y[start:start + size].tobytes()))
    bounds_all = [None] * world
    dist.all_gather_object(bounds_all, b)
    pieces = [None] * world
    dist.all_gather_object(pieces, mine)
    dist.destroy_process_group()
    if rank == 0:
        same = all(x == b for x in bounds_all)
        out = [bytearray(len(c[1].tobytes())) for c in conts]
        written = [0] * len(conts)
        for rp in pieces:
            for i, start, data in rp:
                out[i][start:start + len(data)] = data
                written[i] += len(data)
        ok = all(bytes(out[i]) == conts[i][1].tobytes() for i in range(len(conts)))
        full = all(written[i] == len(out[i]) for i in range(len(conts)))
        q.put((same, ok, full))
    else:
        q.put(None)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_decode_reassembles_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = [r for r in res if r is not None]
    assert got == [(True, True, True)]
