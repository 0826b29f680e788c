"""Periodic-base checkpoint store (ZipNN Sec. 4.2, "Periodic Base").

The policy is checked on the CPU with a byte-level XOR stand-in codec: which
checkpoints are stored whole, what each delta refers to, how long a recovery
chain gets, and that every checkpoint comes back exactly even when the caller
changes its tensors in place after storing them.  On the GPU the same store
runs on the package's codec.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2411_05239_gb300.checkpoint_store import CheckpointStore, GpuCodec


class XorCodec:
    """No compression, only the XOR delta: enough to test the bookkeeping."""

    def compress(self, tensors, bases):
        if bases is None:
            return [np.array(t, dtype=np.uint8).copy() for t in tensors]
        return [np.bitwise_xor(np.asarray(t, np.uint8), np.asarray(b, np.uint8))
                for t, b in zip(tensors, bases)]

    def decompress(self, containers, bases):
        if bases is None:
            return [c.copy() for c in containers]
        return [np.bitwise_xor(c, np.asarray(b, np.uint8)) for c, b in zip(containers, bases)]

    def nbytes(self, containers):
        return sum(int(c.nbytes) for c in containers)


def _run(policy, period, n=23):
    rng = np.random.default_rng(0)
    w = [rng.integers(0, 256, 1000).astype(np.uint8), rng.integers(0, 256, 37).astype(np.uint8)]
    store = CheckpointStore(XorCodec(), period=period, policy=policy)
    history = []
    for _ in range(n):
        store.put(w)
        history.append([x.copy() for x in w])
        for x in w:                       # the "training step" changes the tensors in place
            idx = rng.integers(0, x.size, 5)
            x[idx] ^= rng.integers(1, 256, 5).astype(np.uint8)
    return store, history


@pytest.mark.parametrize("policy", ["chain", "base"])
@pytest.mark.parametrize("period", [1, 5, 10])
def test_every_checkpoint_recovers_exactly(policy, period):
    store, history = _run(policy, period)
    for i, want in enumerate(history):
        got = store.get(i)
        assert all(np.array_equal(g, h) for g, h in zip(got, want)), i


def test_chain_policy_layout():
    store, _ = _run("chain", 10)
    assert [e.is_base for e in store.entries[:12]] == [True] + [False] * 9 + [True, False]
    assert store.entries[7].ref == 6
    assert store.decode_path(9) == list(range(0, 10))      # base + 9 deltas (longest chain)
    assert store.decode_path(10) == [10]
    assert max(len(store.decode_path(i)) for i in range(23)) == 10


def test_base_policy_layout():
    store, _ = _run("base", 10)
    assert store.entries[7].ref == 0 and store.entries[17].ref == 10
    assert all(len(store.decode_path(i)) <= 2 for i in range(23))   # only pairs


def test_bad_arguments():
    with pytest.raises(ValueError):
        CheckpointStore(XorCodec(), period=0)
    with pytest.raises(ValueError):
        CheckpointStore(XorCodec(), policy="zstd")
    store, _ = _run("chain", 5, n=3)
    with pytest.raises(IndexError):
        store.get(3)


@pytest.mark.gpu
@pytest.mark.parametrize("policy", ["chain", "base"])
def test_gpu_store_recovers_checkpoints(policy):
    from paper_2411_05239_gb300 import workloads as W
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    w = [W.gaussian(300_000, 0.02, 1, device="cuda"), W.gaussian(70_001, 0.02, 2, device="cuda")]
    store = CheckpointStore(GpuCodec(), period=4, policy=policy)
    history = []
    for _ in range(9):
        store.put(w)
        history.append([x.clone() for x in w])
        for x in w:   # a small update on 30% of the entries, in place (as c4)
            m = torch.rand(x.numel(), generator=g, device="cuda") < 0.3
            upd = (x.float() + torch.randn(x.numel(), generator=g, device="cuda") * 1e-4).to(x.dtype)
            x.copy_(torch.where(m, upd, x))
    for i, want in enumerate(history):
        got = store.get(i)
        for a, b in zip(got, want):
            assert torch.equal(a.view(torch.int16), b.view(torch.int16)), (policy, i)
    # deltas are much smaller than standalone checkpoints
    full = sum(store.codec.nbytes(e.containers) for e in store.entries if e.is_base)
    dlt = sum(store.codec.nbytes(e.containers) for e in store.entries if not e.is_base)
    nb, nd = sum(e.is_base for e in store.entries), sum(not e.is_base for e in store.entries)
    assert dlt / nd < 0.6 * full / nb
