"""Sharded decoding on the GPU: range plans (needs a GB300).

One GPU plays every rank in turn (ranks never wait on one another, so this is
the same work a rank does on its own GPU): each rank takes its chunk range from
zipnn_partition_chunks, allocates buffers for just its extents, and decodes
them with zipnn_plan_decompress_range; the ranks' bytes, put side by side, must
equal the inputs exactly (lossless, ZipNN Sec. 2.3), whatever the number of
ranks and wherever the cuts fall (mid-tensor, in a delta, in a ragged tail)."""
from __future__ import annotations

import pytest
import torch

from paper_2411_05239_gb300 import workloads as W
from paper_2411_05239_gb300 import zipnn as Z

pytestmark = pytest.mark.gpu

CHUNK = 65536


def _set():
    xs = [W.gaussian(1_000_003, 0.02, 11, device="cuda"),
          torch.ones(4096, dtype=torch.bfloat16, device="cuda"),
          W.gaussian(300_001, 0.05, 12, torch.float32, device="cuda"),
          W.gaussian(700_000, 0.02, 13, torch.float16, device="cuda")]
    nxt, base = W.delta_pair(900_001, seed=14, device="cuda")
    xs.append(nxt)
    bases = [None] * 4 + [base]
    cs = [Z.compress(x, chunk_bytes=CHUNK, base=b) for x, b in zip(xs, bases)]
    return xs, bases, cs


def _maps(cs):
    out = []
    for c in cs:
        P = 64 + 16 * c.zs.n_chunks * c.zs.n_groups
        out.append(c.device_tensor()[:P].cpu())
    return out


@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_ranks_decode_their_ranges_and_reassemble(world):
    xs, bases, cs = _set()
    zss = [c.zs for c in cs]
    b = Z.partition_chunks(zss, _maps(cs), world)
    assert b[0] == 0 and b[-1] == sum(z.n_chunks for z in zss)
    full = [torch.full((x.numel() * x.element_size(),), 0xA5, dtype=torch.uint8, device="cuda")
            for x in xs]
    for r in range(world):
        ext = Z.range_extents(zss, b[r], b[r + 1])
        outs = [torch.empty(e[2], dtype=torch.uint8, device="cuda") if e else None for e in ext]
        rb = [(bases[i].view(torch.uint8)[e[1]:e[1] + e[2]] if (e and bases[i] is not None)
               else None) for i, e in enumerate(ext)]
        pd = Z.plan_decompress_range(cs, outs, b[r], b[r + 1], bases=rb)
        for _ in range(2):                          # plans relaunch
            pd.launch()
        Z.sync_status()
        pd.close()
        for i, e in enumerate(ext):
            if e:
                full[i][e[1]:e[1] + e[2]].copy_(outs[i])
    for x, f in zip(xs, full):
        assert torch.equal(f, x.contiguous().view(-1).view(torch.uint8))


def test_range_arguments_are_checked():
    xs, bases, cs = _set()
    zss = [c.zs for c in cs]
    total = sum(z.n_chunks for z in zss)
    ext = Z.range_extents(zss, 0, total)
    outs = [torch.empty(e[2], dtype=torch.uint8, device="cuda") for e in ext]
    with pytest.raises(Z.ZipnnError):
        Z.plan_decompress_range(cs, outs, 0, total + 1, bases=bases)   # past the end
    with pytest.raises(Z.ZipnnError):
        Z.plan_decompress_range(cs, outs, 3, 3, bases=bases)           # empty range
    with pytest.raises(Z.ZipnnError):
        Z.plan_decompress_range(cs, outs, 0, total, bases=None)        # delta without base
