"""The single-pass encoder (needs a GB300).

On request (encoder option 1), batches of one 16-bit dtype or U8 without the
skip-ahead probe run one persistent kernel per launch: each chunk's histograms, codes, payload offset
(decoupled look-back over the chunks before it in its tensor) and packing.
Its containers must be byte-identical to the four-kernel encoder's and to the
oracle's (ZipNN's container: Sec. 3.1, 3.2, 5.1), including across tensor
boundaries in large batches, empty tensors, ragged tails, every chunk size,
deltas with SPARSE groups, and lane counts that do not divide the chunk; its
bounded wait must give up with ETIMEOUT, leaving the context usable, when a
predecessor never publishes (test-only fault injection)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05239_gb300 import workloads as W
from paper_2411_05239_gb300 import zipnn as Z

pytestmark = pytest.mark.gpu


def u8(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().view(-1).view(torch.uint8).cpu().numpy()


FUSED, SPLIT = 1, 0   # encoder option values


def _run(xs, chunk, encoder, bases=None, lanes=0):
    bc = Z.BatchCompressor(xs, chunk_bytes=chunk, lanes=lanes, bases=bases, encoder=encoder)
    for o in bc.outs:
        o.fill_(0x5A)
    bc()
    Z.sync_status()
    return [c.to_bytes() for c in bc.containers()]


def _batches():
    g = np.random.default_rng(3)
    bf = [W.gaussian(n, 0.02, 100 + i, device="cuda")
          for i, n in enumerate([1, 4097, 131072, 250_001, 0, 70_000, 9, 300_000])]
    bf.append(torch.ones(4096, dtype=torch.bfloat16, device="cuda"))
    bf.append(torch.zeros(5000, dtype=torch.bfloat16, device="cuda"))
    fp = [W.gaussian(n, 0.02, 200 + i, torch.float16, device="cuda")
          for i, n in enumerate([33_333, 262_144, 5])]
    u = [torch.from_numpy(g.geometric(0.3, size=n).clip(0, 255).astype(np.uint8)).cuda()
         for n in (100_003, 16, 65_536)]
    return [("bf16", bf), ("fp16", fp), ("u8", u)]


@pytest.mark.parametrize("chunk", [4096, 16384, 65536, 262144, 1 << 20])
def test_single_pass_equals_four_kernels_and_oracle(chunk):
    for name, xs in _batches():
        fused = _run(xs, chunk, FUSED)
        split = _run(xs, chunk, SPLIT)
        assert fused == split, name
        for x, got in zip(xs, fused):
            assert got == O.compress(u8(x), Z.dtype_code(x, None), chunk), (name, x.numel())


@pytest.mark.parametrize("lanes", [1, 3, 100, 512, 1024])
def test_single_pass_lane_counts(lanes):
    xs = [W.gaussian(n, 0.02, 300 + n, device="cuda") for n in (300_001, 131_072, 77)]
    fused = _run(xs, 262144, FUSED, lanes=lanes)
    assert fused == _run(xs, 262144, SPLIT, lanes=lanes)
    for x, got in zip(xs, fused):
        assert got == O.compress(u8(x), Z.BF16, 262144, lanes)


def test_single_pass_deltas_and_sparse_groups():
    nxt, base = W.delta_pair(600_001, seed=31, device="cuda")
    other = W.gaussian(50_000, 0.02, 32, device="cuda")
    same = W.gaussian(70_000, 0.02, 33, device="cuda")
    xs, bases = [nxt, other, same], [base, None, same]
    fused = _run(xs, 65536, FUSED, bases=bases)
    assert fused == _run(xs, 65536, SPLIT, bases=bases)
    assert fused[0] == O.delta(u8(nxt), u8(base), Z.BF16, 65536)
    assert fused[1] == O.compress(u8(other), Z.BF16, 65536)
    assert fused[2] == O.delta(u8(same), u8(same), Z.BF16, 65536)   # all ZERO


def test_single_pass_many_tensors_one_launch():
    """300 tensors of uneven sizes in one job table: every look-back stops at
    its own tensor's first chunk."""
    rng = np.random.default_rng(9)
    sizes = [int(v) for v in rng.integers(1, 200_000, size=300)]
    xs = [W.gaussian(n, 0.02, 400 + i, device="cuda") for i, n in enumerate(sizes)]
    fused = _run(xs, 16384, FUSED)
    split = _run(xs, 16384, SPLIT)
    assert fused == split
    for i in list(range(0, 300, 37)) + [299]:
        assert fused[i] == O.compress(u8(xs[i]), Z.BF16, 16384)
    # the containers decode back
    cs = [Z.wrap(torch.from_numpy(np.frombuffer(b, dtype=np.uint8).copy()).cuda()) for b in fused]
    outs = [torch.empty_like(x) for x in xs]
    Z.batch_decompress(cs, outs)
    Z.sync_status()
    assert all(torch.equal(x.view(torch.int16), o.view(torch.int16)) for x, o in zip(xs, outs))


def test_lookback_wait_gives_up_with_etimeout_and_context_survives():
    """Fault injection without faulting the GPU: the first chunk never
    publishes its size, so its successors' bounded look-backs give up after
    100 ms (ETIMEOUT); the next call on the same buffers is exact."""
    xs = [W.gaussian(400_000, 0.02, 500, device="cuda"), W.gaussian(9000, 0.02, 501, device="cuda")]
    bc = Z.BatchCompressor(xs, chunk_bytes=65536, encoder=FUSED, debug_flags=1)
    bc()
    with pytest.raises(Z.ZipnnError) as e:
        Z.sync_status()
    assert e.value.status == -5
    good = Z.BatchCompressor(xs, chunk_bytes=65536, encoder=FUSED)
    good()
    Z.sync_status()
    for x, c in zip(xs, good.containers()):
        assert c.to_bytes() == O.compress(u8(x), Z.BF16, 65536)


def test_encoder_options_are_checked():
    x = [W.gaussian(1000, 0.02, 502, device="cuda")]
    with pytest.raises(Z.ZipnnError):
        Z.BatchCompressor(x, chunk_bytes=65536, encoder=2)()
    with pytest.raises(Z.ZipnnError):
        Z.BatchCompressor(x, chunk_bytes=65536, debug_flags=2)()
