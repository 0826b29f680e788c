"""Clean-model workloads (ZipNN Sec. 3.2): parameters held in a wider type than
the precision they carry.

FP32 holding BF16 values has its two low bytes zero, so byte grouping turns
them into all-zero groups that are stored as a header only (the byte-grouping
size table of Sec. 3.2 lists 0.0% for such groups).  FP16 holding BF16 values
has the three low fraction bits of every normal number zero, so among normal
numbers its sign + low-fraction group takes at most 32 byte values and its
entropy stays near 5 bits; the optimal code must land within one bit per symbol
of that entropy.  The CPU tests pin the oracle to these consequences of the
construction; the GPU tests check bit-exactness against it.
"""
from __future__ import annotations

import struct

import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05239_gb300 import workloads as W

CHUNK = 262144


def u8(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().view(-1).view(torch.uint8).cpu().numpy()


def entries(stream: bytes):
    G = struct.unpack_from("<I", stream, 24)[0]
    nch = struct.unpack_from("<I", stream, 28)[0]
    T = struct.unpack_from("<I", stream, 20)[0]
    ent = [struct.unpack_from("<QIBB", stream, 64 + 16 * i) for i in range(nch * G)]
    return G, nch, T, ent


def test_clean_fp32_low_groups_are_zero_and_exponent_is_huffman():
    x = W.clean_fp32_from_bf16(1_048_576 + 3, seed=5)
    xs = u8(x)
    s = O.compress(xs, O.FP32, CHUNK)
    G, nch, T, ent = entries(s)
    assert G == 4 and nch == 17
    for c in range(nch):
        modes = [ent[c * G + g][2] for g in range(G)]
        assert modes[2] == 2 and modes[3] == 2, (c, modes)    # ZERO: header only
        assert ent[c * G + 2][1] == 0 and ent[c * G + 3][1] == 0
        if c < nch - 1:
            assert modes[0] == 1                                # exponent: HUFF
    # two of four bytes vanish, the exponent group compresses to about a third
    assert 0.30 < len(s) / xs.size < 0.36
    assert np.array_equal(O.decompress(s), xs)


def test_clean_fp16_fraction_group_within_entropy_bounds():
    x = W.clean_fp16_from_bf16(1_048_576, seed=6)
    xs = u8(x)
    v = xs.view(np.uint16)
    # the construction: every normal FP16 value has its 3 low fraction bits zero
    normal = ((v >> 10) & 0x1F) != 0
    assert np.all((v[normal] & 7) == 0)
    # group 1 = sign + low 7 fraction bits, computed here with plain bit operations
    g1 = (((v >> 8) & 0x80) | (v & 0x7F)).astype(np.int64)
    s = O.compress(xs, O.FP16, CHUNK)
    G, nch, T, ent = entries(s)
    P = struct.unpack_from("<Q", s, 32)[0]
    m = CHUNK // 2
    for c in range(nch):
        off, size, mode, value = ent[c * G + 1]
        assert mode == 1, c
        cnt = np.bincount(g1[c * m:(c + 1) * m], minlength=256)
        p = cnt[cnt > 0] / m
        H = float(-(p * np.log2(p)).sum())
        assert H < 5.2            # 32 normal symbols plus a few subnormal ones
        nz = int(np.count_nonzero(cnt))
        pay = s[P + off: P + off + size]
        assert sum(pay[:12]) == nz
        h = (12 + nz + 3) // 4 * 4 + 4 * (T - 1)
        # optimal prefix code: n*H <= bits < n*(H + 1); the bitstream is whole words
        nbits_max = 32 * ((size - h) // 4)
        assert m * H <= nbits_max < m * (H + 1) + 32, (c, H, nbits_max)
    assert np.array_equal(O.decompress(s), xs)


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["fp32", "fp16"])
@pytest.mark.parametrize("n", [1_048_576 + 5, 3_000_000])
def test_clean_models_gpu_identical_to_oracle(which, n):
    from paper_2411_05239_gb300 import zipnn as Z
    if which == "fp32":
        x, dt = W.clean_fp32_from_bf16(n, seed=7, device="cuda"), O.FP32
    else:
        x, dt = W.clean_fp16_from_bf16(n, seed=8, device="cuda"), O.FP16
    xs = u8(x)
    c = Z.compress(x)
    assert c.to_bytes() == O.compress(xs, dt, CHUNK)
    y = Z.decompress(c)
    Z.sync_status()
    assert np.array_equal(u8(y), xs)


@pytest.mark.gpu
def test_clean_models_full_size_round_trip():
    from paper_2411_05239_gb300 import zipnn as Z
    for make in (W.clean_fp32_from_bf16, W.clean_fp16_from_bf16):
        x = make(device="cuda")
        dt = Z.dtype_code(x, None)
        c = Z.compress(x)
        out = torch.empty_like(x)
        Z.batch_decompress([c], [out])
        Z.sync_status()
        assert torch.equal(out.view(torch.uint8), x.view(torch.uint8))
        # sampled chunks: payloads identical to the oracle's encoding of them
        t = c.to_bytes()
        G, nch, T, ent = entries(t)
        P = struct.unpack_from("<Q", t, 32)[0]
        xb = x.view(torch.uint8)
        for ch in (0, nch // 2, nch - 1):
            want = O.compress_chunk(xb[ch * CHUNK:(ch + 1) * CHUNK].cpu().numpy(), dt, T)
            for g in range(G):
                off, size, mode, value = ent[ch * G + g]
                assert (mode, value, size) == (want[g][0], want[g][1], len(want[g][2]))
                assert t[P + off: P + off + size] == want[g][2]
