"""Skip-ahead probe (ZipNN Sec. 3.2, "Identifying compressibility").

The paper compresses a chunk and, when it is not compressible, does not try the
following few chunks before trying again.  With probe_skip = k: after a
group-chunk decided raw, the same group of the next k chunks is stored raw, then
decisions resume.  The CPU tests pin the oracle's mode sequences to sequences
worked out by hand from that rule (one per line below, with the derivation);
the GPU tests require byte-identical containers from the batched encoder.
"""
from __future__ import annotations

import struct

import numpy as np
import pytest
import torch

import oracle as O

CHUNK = 4096


def modes_of(stream: bytes) -> str:
    G = struct.unpack_from("<I", stream, 24)[0]
    nch = struct.unpack_from("<I", stream, 28)[0]
    name = {0: "R", 1: "H", 2: "Z", 3: "C"}
    return "".join(name[stream[64 + 16 * (c * G + g) + 12]] for c in range(nch) for g in range(G))


def pattern_u8(pattern: str, seed: int = 0) -> np.ndarray:
    """One 4096-byte U8 chunk per letter: 'C' compressible (bytes 1 and 2 in a
    9:1 mix: Huffman), 'I' incompressible (uniform random bytes: raw)."""
    g = np.random.default_rng(seed)
    parts = []
    for p in pattern:
        if p == "C":
            parts.append(np.where(g.random(CHUNK) < 0.9, 1, 2).astype(np.uint8))
        else:
            parts.append(g.integers(0, 256, CHUNK).astype(np.uint8))
    return np.concatenate(parts)


CASES = [
    # k = 0: every chunk decided on its own
    ("CICCCICC", 0, "HRHHHRHH"),
    # k = 1: c1 raw -> c2 skipped; c3, c4 decided; c5 raw -> c6 skipped; c7 decided
    ("CICCCICC", 1, "HRRHHRRH"),
    # k = 2: c1 raw -> c2, c3 skipped; c4 decided; c5 raw -> c6, c7 skipped
    ("CICCCICC", 2, "HRRRHRRR"),
    # k = 2: c0 raw -> c1, c2 skipped; c3 .. c7 decided
    ("IIICCCCC", 2, "RRRHHHHH"),
    # k = 1: c0, c2, c4, c6 decided raw, each skipping the compressible chunk after it
    ("ICICICIC", 1, "RRRRRRRR"),
    # k = 3: skipping after c4 only covers chunks that are raw anyway
    ("CCCCIIII", 3, "HHHHRRRR"),
    # k = 2: c1 raw -> c2, c3 skipped; c4 decided raw -> c5 (compressible) skipped
    ("CIIIIC", 2, "HRRRRR"),
]


@pytest.mark.parametrize("pattern,k,want", CASES)
def test_oracle_mode_sequences(pattern, k, want):
    x = pattern_u8(pattern)
    s = O.compress(x, O.U8, CHUNK, 8, skip=k)
    assert modes_of(s) == want
    assert np.array_equal(O.decompress(s), x)


def test_skipped_chunks_hold_their_raw_bytes():
    x = pattern_u8("CICCCICC")
    s = O.compress(x, O.U8, CHUNK, 8, skip=2)
    P = struct.unpack_from("<Q", s, 32)[0]
    for c in (2, 3):                                    # compressible, but skipped
        off, size, mode = struct.unpack_from("<QIB", s, 64 + 16 * c)
        assert mode == 0 and size == CHUNK
        assert s[P + off: P + off + size] == x[c * CHUNK:(c + 1) * CHUNK].tobytes()


def test_skip_changes_nothing_on_model_weights():
    """BF16 weights: the exponent group is never raw and the sign + fraction
    group always is, so skipping never changes a decision."""
    t = torch.randn(1 << 19, generator=torch.Generator().manual_seed(3)) * 0.02
    x = t.to(torch.bfloat16).view(torch.uint8).numpy()
    assert O.compress(x, O.BF16, 65536, skip=4) == O.compress(x, O.BF16, 65536)


def bf16_turning_compressible(n: int = 1 << 16) -> torch.Tensor:
    """BF16 weights whose second half has its 7 low fraction bits cleared: the
    sign + fraction group is raw in the first half, Huffman in the second."""
    w = (torch.randn(n, generator=torch.Generator().manual_seed(4)) * 0.02).to(torch.bfloat16)
    w[n // 2:] = w[n // 2:].view(torch.int16).bitwise_and(~0x7F).view(torch.bfloat16)
    return w


def test_window_spills_into_a_compressible_region():
    """Chunks 0-15 of the second group are incompressible, 16-31 compressible.
    With k = 5 the chunks decided are 0, 6 and 12 (each raw, each opening a
    window of 5), so chunks 16 and 17 lie in the window of chunk 12 and are
    stored raw; chunk 18 is decided again (Huffman).  With k = 3 the decided
    chunks are 0, 4, 8, 12, whose last window ends at chunk 15: nothing spills."""
    x = bf16_turning_compressible().view(torch.uint8).numpy()
    m = modes_of(O.compress(x, O.BF16, CHUNK, 8, skip=5))
    assert m[1::2] == "R" * 18 + "H" * 14
    assert m[0::2] == "H" * 32
    m = modes_of(O.compress(x, O.BF16, CHUNK, 8, skip=3))
    assert m[1::2] == "R" * 16 + "H" * 16


@pytest.mark.gpu
@pytest.mark.parametrize("k", [0, 1, 2, 5])
def test_gpu_probe_skip_identical_to_oracle(k):
    from paper_2411_05239_gb300 import zipnn as Z
    xs = [pattern_u8("CICCCICCIIICCCCCICIC", seed=1), pattern_u8("CCIC", seed=2)[:CHUNK * 3 + 100]]
    bufs = [torch.from_numpy(x).cuda() for x in xs] + [bf16_turning_compressible().cuda()]
    bc = Z.BatchCompressor(bufs, chunk_bytes=CHUNK, lanes=8, probe_skip=k)
    bc()
    Z.sync_status()
    cs = bc.containers()
    for c, b, dt in zip(cs, bufs, [O.U8, O.U8, O.BF16]):
        want = O.compress(b.view(torch.uint8).cpu().numpy(), dt, CHUNK, 8, skip=k)
        assert c.to_bytes() == want
        y = Z.decompress(c)
        Z.sync_status()
        assert torch.equal(y.view(torch.uint8).cpu(), b.view(torch.uint8).cpu())
