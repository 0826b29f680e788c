"""Load plan (zipnn_plan_load) vs the inputs (needs a GB300).

Containers kept in pinned host memory are copied to the device and decoded
segment by segment, copies and decoding overlapped, in one CUDA graph.  The
decoded bytes must equal the original tensors (lossless, ZipNN Sec. 2.3), for
every segment split, repeatedly, including delta containers (Sec. 4.2).
"""
from __future__ import annotations

import pytest
import torch

from paper_2411_05239_gb300 import workloads as W
from paper_2411_05239_gb300 import zipnn as Z

pytestmark = pytest.mark.gpu


def _setup():
    xs = [W.gaussian(n, 0.02, 100 + i) for i, n in enumerate([1_000_003, 262_144, 5, 2_500_000])]
    xs.append(W.gaussian(300_001, 0.05, 110, torch.float32))
    xs = [x.cuda() for x in xs]
    nxt, base = W.delta_pair(700_000, seed=111, device="cuda")
    cs = [Z.compress(x) for x in xs] + [Z.compress(nxt, base=base)]
    ys = xs + [nxt]
    bases = [None] * len(xs) + [base]
    return cs, ys, bases


@pytest.mark.parametrize("segment_bytes", [0, 1, 300_000])
def test_load_plan_decodes_host_containers(segment_bytes):
    cs, ys, bases = _setup()
    h = [torch.empty(c.nbytes, dtype=torch.uint8, pin_memory=True) for c in cs]
    for hc, c in zip(h, cs):
        hc.copy_(c.device_tensor())
    torch.cuda.synchronize()
    # the device containers are overwritten by every launch: start from zeros
    for c in cs:
        c.device_tensor().zero_()
    outs = [torch.empty_like(y) for y in ys]
    plan = Z.plan_load(cs, h, outs, bases=bases, segment_bytes=segment_bytes)
    for _ in range(2):
        for o in outs:
            o.zero_()
        plan.launch()
        Z.sync_status()
        for y, o in zip(ys, outs):
            assert torch.equal(o.view(torch.uint8), y.view(torch.uint8))
    plan.close()


def test_load_plan_rejects_pageable_host_memory():
    cs, ys, bases = _setup()
    h = [torch.empty(c.nbytes, dtype=torch.uint8) for c in cs]
    with pytest.raises(ValueError):
        Z.plan_load(cs, h, [torch.empty_like(y) for y in ys], bases=bases)


@pytest.mark.parametrize("segment_bytes", [0, 300_000])
def test_load_plan_coalesces_adjacent_containers_only(segment_bytes):
    """Containers back to back in both a pinned host arena and a device arena
    go over in one copy per run; a gap on either side splits the run, and the
    device bytes in a gap are never written."""
    cs, ys, bases = _setup()
    n = len(cs)
    gap = 32
    # device gap after container 1, host gap after container 3
    dgap = [gap if i == 1 else 0 for i in range(n)]
    hgap = [gap if i == 3 else 0 for i in range(n)]
    hoff, doff, ho, do = [], [], 0, 0
    for i, c in enumerate(cs):
        assert c.nbytes % 16 == 0
        hoff.append(ho)
        doff.append(do)
        ho += c.nbytes + hgap[i]
        do += c.nbytes + dgap[i]
    harena = torch.full((ho,), 0xA5, dtype=torch.uint8, pin_memory=True)
    darena = torch.full((do,), 0x3C, dtype=torch.uint8, device="cuda")
    for i, c in enumerate(cs):
        harena[hoff[i]:hoff[i] + c.nbytes].copy_(c.device_tensor())
    torch.cuda.synchronize()
    lcs = []
    for i, c in enumerate(cs):
        dv = darena[doff[i]:doff[i] + c.nbytes]
        dv.copy_(c.device_tensor())
        lcs.append(Z.wrap(dv, c.nbytes))
    for i, c in enumerate(cs):   # the load must bring every container byte
        darena[doff[i]:doff[i] + c.nbytes].zero_()
    hs = [harena[hoff[i]:hoff[i] + c.nbytes] for i, c in enumerate(cs)]
    outs = [torch.empty_like(y) for y in ys]
    plan = Z.plan_load(lcs, hs, outs, bases=bases, segment_bytes=segment_bytes)
    for _ in range(2):
        for o in outs:
            o.zero_()
        plan.launch()
        Z.sync_status()
        for y, o in zip(ys, outs):
            assert torch.equal(o.view(torch.uint8), y.view(torch.uint8))
        g0 = doff[1] + cs[1].nbytes
        assert torch.all(darena[g0:g0 + gap] == 0x3C)
    plan.close()
