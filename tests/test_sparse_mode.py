"""SPARSE group mode: Huffman over the vectors that hold a non-zero symbol,
plus a bitmap of those vectors.  It stands in for the paper's switch from
Huffman to Zstd on delta chunks that are mostly zeros (ZipNN Sec. 4.2, "Auto
Detection"): Huffman alone spends at least one bit per symbol.

The CPU tests pin the oracle to facts outside it: the one-bit floor of a
prefix code (a mostly-zero delta exponent group coded below m/8 bytes can only
come from leaving the zero vectors out), the entropy bounds of an optimal code
on the histogram of the coded symbols (computed here with numpy), the bitmap
size, and lossless round trips; the GPU tests require byte-identical
containers and exact decoding.
"""
from __future__ import annotations

import struct

import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05239_gb300 import workloads as W
from tests import spec_decoder

CHUNK = 262144


def groups_bf16(x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Byte groups of BF16 data with plain bit operations (exponent byte; sign +
    low 7 fraction bits)."""
    v = x.view(np.uint16)
    return ((v >> 7) & 0xFF).astype(np.uint8), (((v >> 8) & 0x80) | (v & 0x7F)).astype(np.uint8)


def entries(s: bytes):
    G = struct.unpack_from("<I", s, 24)[0]
    nch = struct.unpack_from("<I", s, 28)[0]
    T = struct.unpack_from("<I", s, 20)[0]
    P = struct.unpack_from("<Q", s, 32)[0]
    return G, nch, T, P, [struct.unpack_from("<QIBB", s, 64 + 16 * i) for i in range(nch * G)]


def delta_bytes(n: int, seed: int):
    nxt, base = W.delta_pair(n, seed=seed)
    return nxt.view(torch.uint8).numpy(), base.view(torch.uint8).numpy()


def test_delta_exponent_group_beats_the_one_bit_floor():
    a, b = delta_bytes(1 << 20, 3)
    s = O.delta(a, b, O.BF16, CHUNK)
    G, nch, T, P, ent = entries(s)
    m = CHUNK // 2
    for c in range(nch):
        off, size, mode, value = ent[c * G]
        assert mode == 4                     # SPARSE
        assert size < m // 8                 # below what any per-symbol prefix code needs
    assert np.array_equal(O.decompress(s, b), a)
    assert spec_decoder.decode(s, b.tobytes()) == a.tobytes()


def test_sparse_payload_layout_and_entropy_bounds():
    a, b = delta_bytes(1 << 20, 4)
    d = np.bitwise_xor(a, b)
    s = O.delta(a, b, O.BF16, CHUNK)
    G, nch, T, P, ent = entries(s)
    m, V = CHUNK // 2, 8
    g0, g1 = groups_bf16(d)
    for c in range(nch):
        for g, plane in ((0, g0), (1, g1)):
            off, size, mode, value = ent[c * G + g]
            if mode != 4:
                continue
            sym = plane[c * m:(c + 1) * m]
            nonzero = sym.reshape(-1, V).any(axis=1)
            coded = sym.reshape(-1, V)[nonzero].reshape(-1)
            cnt = np.bincount(coded, minlength=256)
            p = cnt[cnt > 0] / coded.size
            H = float(-(p * np.log2(p)).sum())
            pay = s[P + off: P + off + size]
            nz = sum(pay[:12])
            assert nz == np.count_nonzero(cnt)
            h = (12 + nz + 3) // 4 * 4
            nbw = (m // V + 31) // 32
            bitmap = np.frombuffer(pay[h:h + 4 * nbw], dtype=np.uint8)
            assert np.array_equal(np.unpackbits(bitmap, bitorder="little")[: m // V], nonzero)
            nbits_max = 32 * ((size - h - 4 * nbw - 4 * (T - 1)) // 4)
            assert coded.size * H <= nbits_max < coded.size * (H + 1) + 32
    assert np.array_equal(O.decompress(s, b), a)


def test_pruned_weights_take_sparse_and_round_trip():
    """Weights with 90% of the values pruned to exactly zero in blocks of 8."""
    g = np.random.default_rng(5)
    w = (g.standard_normal(1 << 19) * 0.02).astype(np.float32)
    keep = np.repeat(g.random((1 << 19) // 8) < 0.1, 8)
    x = torch.from_numpy(np.where(keep, w, 0).astype(np.float32)).to(torch.bfloat16)
    xs = x.view(torch.uint8).numpy()
    s = O.compress(xs, O.BF16, CHUNK)
    G, nch, T, P, ent = entries(s)
    assert all(e[2] == 4 for e in ent)
    assert len(s) < 0.2 * xs.size
    assert np.array_equal(O.decompress(s), xs)
    assert spec_decoder.decode(s) == xs.tobytes()


def test_weights_without_zero_vectors_never_take_sparse():
    x = W.gaussian(1 << 19, 0.02, 6).view(torch.uint8).numpy()
    s = O.compress(x, O.BF16, CHUNK)
    assert all(e[2] in (0, 1) for e in entries(s)[4])


@pytest.mark.gpu
@pytest.mark.parametrize("lanes", [0, 8, 256, 512])
def test_gpu_sparse_identical_to_oracle(lanes):
    from paper_2411_05239_gb300 import zipnn as Z
    nxt, base = W.delta_pair(1_300_007, seed=7, device="cuda")
    c = Z.compress(nxt, base=base, lanes=lanes)
    a, b = nxt.view(torch.uint8).cpu().numpy(), base.view(torch.uint8).cpu().numpy()
    assert c.to_bytes() == O.delta(a, b, O.BF16, CHUNK, lanes or None)
    out = torch.empty_like(nxt)
    Z.batch_decompress([c], [out], bases=[base])
    Z.sync_status()
    assert torch.equal(out.view(torch.int16), nxt.view(torch.int16))
    g = np.random.default_rng(8)
    w = (g.standard_normal(600_000) * 0.02).astype(np.float32)
    keep = np.repeat(g.random(75_000) < 0.1, 8)
    x = torch.from_numpy(np.where(keep, w, 0).astype(np.float32)).to(torch.bfloat16).cuda()
    c = Z.compress(x, lanes=lanes)
    assert c.to_bytes() == O.compress(x.view(torch.uint8).cpu().numpy(), O.BF16, CHUNK, lanes or None)
    y = Z.decompress(c)
    Z.sync_status()
    assert torch.equal(y.view(torch.int16), x.view(torch.int16))
