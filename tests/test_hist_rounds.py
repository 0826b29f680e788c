"""FP32 histograms with packed 16-bit counters, counted in rounds (needs a GB300).

The FP32 histogram keeps two 16-bit counters per shared-memory word and
counts a chunk in rounds of 4 MiB of vectors, each round folded into 32-bit
totals before the counters could overflow.  The containers must equal the
oracle's byte for byte (ZipNN Sec. 3.1, 3.2: the codes follow the exact
histograms) for chunks of one round and of several, for a symbol that fills
nearly every vector (one counter word would pass 2^16 without the rounds),
alone and in a batch with 16-bit tensors (the mixed-dtype kernel).
"""
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


def skewed_fp32(n: int, seed: int) -> torch.Tensor:
    """90% of the values exactly 0.75, the rest N(0, 0.05)."""
    g = np.random.default_rng(seed)
    x = (g.standard_normal(n) * 0.05).astype(np.float32)
    x[g.random(n) < 0.9] = 0.75
    return torch.from_numpy(x)


@pytest.mark.parametrize("chunk", [16 << 20, 8 << 20, (4 << 20) + 4096, 262144])
def test_fp32_histogram_rounds(chunk):
    xs = [skewed_fp32(5_000_003, 130), W.gaussian(4_500_001, 0.05, 131, torch.float32)]
    for x in xs:
        c = Z.compress(x.cuda(), chunk_bytes=chunk)
        assert c.to_bytes() == O.compress(u8(x), Z.FP32, chunk), chunk
        y = Z.decompress(c)
        Z.sync_status()
        assert torch.equal(y.cpu().view(torch.int32), x.view(torch.int32))


def test_fp32_histogram_in_a_mixed_batch():
    xs = [skewed_fp32(3_000_001, 132), W.gaussian(1_000_003, 0.02, 133),
          W.gaussian(700_001, 0.02, 134, torch.float16), skewed_fp32(2_000_000, 135)]
    chunk = 8 << 20
    bc = Z.BatchCompressor([x.cuda() for x in xs], chunk_bytes=chunk)
    bc()
    Z.sync_status()
    for x, c in zip(xs, bc.containers()):
        assert c.to_bytes() == O.compress(u8(x), Z.dtype_code(x, None), chunk)
