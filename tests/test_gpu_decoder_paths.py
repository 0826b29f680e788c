"""Decoder launch shapes and loops vs the CPU oracle (needs a GB300).

The decoder has a specialised loop for chunks whose exponent group is Huffman
coded and whose other groups are raw, zero or constant, and a generic loop for
everything else; it runs with 128- or 256-thread CTAs, one or two sub-streams
per thread, and W = 10, 11 or 12 bit pair tables (W = 11 resolves 12-bit codes
inside the table entry).  None of these choices may change a decoded byte
(lossless, ZipNN Sec. 2.3), and every container must stay byte-identical to the
oracle's (Sec. 3.1, 3.2 and 5.1 as specified for the container).
"""
from __future__ import annotations

import struct

import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05239_gb300 import workloads as W
from paper_2411_05239_gb300 import zipnn as Z

pytestmark = pytest.mark.gpu


def u8(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().view(-1).view(torch.uint8).cpu().numpy()


def skewed_exponents_bf16(n: int, seed: int) -> torch.Tensor:
    """BF16 values whose exponent byte e = 0x7F - k has P(k) ~ 2^-k (k < 40):
    the length limit of 12 binds, so every chunk holds codes of 11 and 12 bits."""
    g = np.random.default_rng(seed)
    k = np.minimum(g.geometric(0.5, size=n) - 1, 39)
    e = (0x7F - k).astype(np.uint16)
    frac = g.integers(0, 128, size=n).astype(np.uint16)
    sign = (g.random(n) < 0.5).astype(np.uint16) << 15
    bits = sign | (e << 7) | frac
    return torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16)


def max_code_len(stream: bytes) -> int:
    """Longest code length of any Huffman group-chunk in a container."""
    P = struct.unpack_from("<Q", stream, 32)[0]
    G = struct.unpack_from("<I", stream, 24)[0]
    nch = struct.unpack_from("<I", stream, 28)[0]
    best = 0
    for i in range(nch * G):
        off, size, mode = struct.unpack_from("<QIB", stream, 64 + 16 * i)
        if mode == 1:
            bits = stream[P + off: P + off + 12]
            best = max(best, max(l + 1 for l in range(12) if bits[l]))
    return best


CASES = [
    ("bf16_gauss", Z.BF16, lambda: W.gaussian(600_001, 0.02, 81)),
    ("bf16_long_codes", Z.BF16, lambda: skewed_exponents_bf16(524_288 + 77, 82)),
    ("fp32_clean", Z.FP32, lambda: W.clean_fp32_from_bf16(262_144 + 5, 83)),
    ("fp32_gauss", Z.FP32, lambda: W.gaussian(262_144, 0.05, 84, torch.float32)),
    ("fp16_from_bf16", Z.FP16, lambda: W.clean_fp16_from_bf16(300_000, 85)),
    ("u8_skewed", Z.U8, lambda: torch.from_numpy(
        np.random.default_rng(86).geometric(0.3, size=1_048_576 + 9).clip(0, 255).astype(np.uint8))),
]


@pytest.mark.parametrize("name,dtype,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("lanes", [128, 256, 512, 768])
def test_cta_sizes_table_widths_and_lanes(name, dtype, make, lanes):
    x = make()
    xs = u8(x)
    chunk = 262144
    c = Z.compress(x.cuda(), chunk_bytes=chunk, lanes=lanes, dtype=dtype)
    want = O.compress(xs, dtype, chunk, lanes)
    assert c.to_bytes() == want
    out = torch.empty_like(x, device="cuda")
    for w in (10, 11, 12):
        for nt in (128, 256):
            out.zero_()
            Z.batch_decompress([c], [out], tune=Z.tuning(threads=nt, lut_bits=w))
            Z.sync_status()
            assert np.array_equal(u8(out), xs), (w, nt)


def test_long_codes_are_present():
    """The skewed case really exercises 12-bit codes (the W = 11 long entries)."""
    x = skewed_exponents_bf16(262_144, 90)
    assert max_code_len(O.compress(u8(x), Z.BF16, 262144)) == 12


@pytest.mark.parametrize("lanes", [256, 512])
def test_delta_on_fast_loop(lanes):
    n = 524_288
    nxt, base = W.delta_pair(n, seed=91, device="cuda")
    c = Z.compress(nxt, chunk_bytes=262144, lanes=lanes, base=base)
    assert c.to_bytes() == O.delta(u8(nxt), u8(base), Z.BF16, 262144, lanes)
    out = torch.empty_like(nxt)
    for nt in (128, 256):
        Z.batch_decompress([c], [out], bases=[base], tune=Z.tuning(threads=nt))
        Z.sync_status()
        assert torch.equal(out.view(torch.int16), nxt.view(torch.int16))


def test_mixed_batch_of_all_layouts():
    """One persistent launch over tensors that take different loops and dtypes."""
    xs = [make() for _, _, make in CASES]
    cs = [Z.compress(x.cuda(), chunk_bytes=131072, lanes=256) for x in xs]
    outs = [torch.empty_like(x, device="cuda") for x in xs]
    Z.batch_decompress(cs, outs)
    Z.sync_status()
    for x, o in zip(xs, outs):
        assert np.array_equal(u8(o), u8(x))


def test_wrong_substream_start_reports_ecorrupt_and_context_survives():
    """A start-bit entry moved by one bit breaks the rule that every sub-stream
    ends where the next one begins: the chunk is reported corrupt."""
    x = W.gaussian(262_144 * 4, 0.02, 92)
    c = Z.compress(x.cuda(), chunk_bytes=262144, lanes=256)
    s = bytearray(c.to_bytes())
    P = struct.unpack_from("<Q", s, 32)[0]
    off, size, mode = struct.unpack_from("<QIB", s, 64 + 16 * (2 * 2))   # chunk 2, group 0
    assert mode == 1
    nz = sum(s[P + off: P + off + 12])
    h = (12 + nz + 3) // 4 * 4
    p = P + off + h + 4 * 4          # start bit of sub-stream 5
    struct.pack_into("<I", s, p, struct.unpack_from("<I", s, p)[0] + 1)
    buf = torch.from_numpy(np.frombuffer(bytes(s), dtype=np.uint8).copy()).cuda()
    bad = Z.wrap(buf)
    out = torch.empty_like(x, device="cuda")
    Z.batch_decompress([bad], [out])
    with pytest.raises(Z.ZipnnError) as ei:
        Z.sync_status()
    assert ei.value.status == -3  # ZIPNN_ECORRUPT
    # the context still works
    y = Z.decompress(c)
    Z.sync_status()
    assert torch.equal(y.cpu().view(torch.int16), x.view(torch.int16))


def pruned_bf16(n: int, seed: int) -> torch.Tensor:
    """BF16 weights with 90% of their 16-byte vectors zero: SPARSE groups."""
    g = np.random.default_rng(seed)
    w = (g.standard_normal(n) * 0.02).astype(np.float32)
    keep = np.repeat(g.random((n + 7) // 8) < 0.1, 8)[:n]
    return torch.from_numpy(np.where(keep, w, 0).astype(np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("with_delta", [False, True])
@pytest.mark.parametrize("mixed_dtypes", [False, True])
def test_batches_with_and_without_deltas(with_delta, mixed_dtypes):
    """A launch that holds a delta runs the kernels with the general fast loops
    (two coded groups, SPARSE bitmaps); every other stream of that launch must
    decode through them as well, and without a delta the same streams take the
    Huffman loop of model weights and the generic loop."""
    xs = [W.gaussian(700_000, 0.02, 93), pruned_bf16(600_000, 94),
          skewed_exponents_bf16(524_288, 95)]
    if mixed_dtypes:
        xs += [W.clean_fp16_from_bf16(300_000, 96), W.clean_fp32_from_bf16(262_144, 97)]
    cs = [Z.compress(x.cuda()) for x in xs]
    for c, x in zip(cs, xs):
        assert c.to_bytes() == O.compress(u8(x), Z.dtype_code(x, None), Z.DEFAULT_CHUNK)
    bases = [None] * len(xs)
    if with_delta:
        nxt, base = W.delta_pair(900_001, seed=98, device="cuda")
        c = Z.compress(nxt, base=base)
        assert c.to_bytes() == O.delta(u8(nxt), u8(base), Z.BF16, Z.DEFAULT_CHUNK)
        xs, cs, bases = xs + [nxt], cs + [c], bases + [base]
    outs = [torch.empty_like(x, device="cuda") for x in xs]
    for nt in (128, 256):
        for o in outs:
            o.zero_()
        Z.batch_decompress(cs, outs, bases=bases, tune=Z.tuning(threads=nt))
        Z.sync_status()
        for x, o in zip(xs, outs):
            assert np.array_equal(u8(o), u8(x)), nt


def _modes(stream: bytes, chunk: int) -> list[tuple[int, int]]:
    G = struct.unpack_from("<I", stream, 24)[0]
    return [tuple(stream[64 + 16 * (chunk * G + g) + 12: 64 + 16 * (chunk * G + g) + 14])
            for g in range(G)]


@pytest.mark.parametrize("pattern", ["fp32_const_low", "fp32_zero_mid", "bf16_const_low"])
def test_fast_loops_with_constant_and_zero_groups(pattern):
    """The fast loops read raw groups through a per-thread shared-memory ring
    (FP32) or registers (16-bit), prefetched into L2 by the chunk's window;
    ZERO and CONST groups come from the map's value byte instead.  Three full
    256 KiB chunks plus a ragged one, every CTA size and table width."""
    if pattern.startswith("fp32"):
        x = W.gaussian(3 * 65536 + 1000, 0.05, 99, torch.float32)
        b = x.view(torch.int32)
        b = (b & ~0xFF) | 0x5A if pattern == "fp32_const_low" else b & ~0xFF00
        x, dt = b.view(torch.float32), Z.FP32
        want_mode = (3, 0x5A) if pattern == "fp32_const_low" else (2, 0)
        g_const = 3 if pattern == "fp32_const_low" else 2
    else:
        g = np.random.default_rng(100)
        e = (0x7F - np.minimum(g.geometric(0.5, size=3 * 131072 + 777) - 1, 20)).astype(np.uint16)
        x = torch.from_numpy(((e << 7) | 0x2A).view(np.int16)).view(torch.bfloat16)
        dt, want_mode, g_const = Z.BF16, (3, 0x2A), 1
    xs = u8(x)
    c = Z.compress(x.cuda())
    s = c.to_bytes()
    assert s == O.compress(xs, dt, Z.DEFAULT_CHUNK)
    for ch in range(3):
        m = _modes(s, ch)
        assert m[0][0] == 1 and m[g_const] == want_mode, (ch, m)
    out = torch.empty_like(x, device="cuda")
    for nt in (128, 256):
        for w in (11, 12):
            out.zero_()
            Z.batch_decompress([c], [out], tune=Z.tuning(threads=nt, lut_bits=w))
            Z.sync_status()
            assert np.array_equal(u8(out), xs), (nt, w)


@pytest.mark.parametrize("which", ["clean_fp16", "pruned_bf16", "clean_fp16_and_gauss"])
def test_plans_size_their_stage_from_the_chunk_maps(which):
    """A decode plan reads its containers' chunk maps: FP16 holding BF16
    values codes both byte groups (about 170 KiB per 256 KiB chunk, more than
    the default stage), so the plan stages them with one CTA per SM and runs
    the two-group loop; pruned BF16 has SPARSE exponent groups.  Plans and load
    plans must decode every byte as the direct calls do."""
    if which == "clean_fp16":
        xs = [W.clean_fp16_from_bf16(3 * 131072 + 999, 110)]
    elif which == "pruned_bf16":
        xs = [pruned_bf16(4 * 131072, 111)]
    else:
        xs = [W.clean_fp16_from_bf16(2 * 131072, 112), W.gaussian(3 * 131072 + 5, 0.02, 113,
                                                                   torch.float16)]
    cs = [Z.compress(x.cuda()) for x in xs]
    for c, x in zip(cs, xs):
        assert c.to_bytes() == O.compress(u8(x), Z.dtype_code(x, None), Z.DEFAULT_CHUNK)
    outs = [torch.empty_like(x, device="cuda") for x in xs]
    for nt in (128, 256):
        for o in outs:
            o.zero_()
        p = Z.plan_decompress(cs, outs, tune=Z.tuning(threads=nt))
        p.launch()
        Z.sync_status()
        p.close()
        for x, o in zip(xs, outs):
            assert np.array_equal(u8(o), u8(x)), nt
    h = [torch.from_numpy(np.frombuffer(c.to_bytes(), dtype=np.uint8).copy()).pin_memory()
         for c in cs]
    for o in outs:
        o.zero_()
    p = Z.plan_load(cs, h, outs)
    p.launch()
    Z.sync_status()
    p.close()
    for x, o in zip(xs, outs):
        assert np.array_equal(u8(o), u8(x))


@pytest.mark.parametrize("parts", [0, 1, 2, 4, 8])
def test_chunks_split_over_work_items_decode_the_same(parts):
    """Launches with few chunks split each model-weight chunk's sub-streams
    over 2, 4 or 8 work items (tuning.parts: 0 = automatic); chunks of other
    layouts (ragged last chunk, FP32, lanes that do not split) are decoded
    whole by their first part.  The decoded bytes never change."""
    xs = [W.plain_bf16(device="cuda"),                                   # 32 full chunks
          W.gaussian(300_001, 0.02, 81, device="cuda"),                  # ragged tail
          W.gaussian(1 << 19, 0.02, 82, torch.float16, device="cuda"),
          W.gaussian(700_000, 0.05, 83, torch.float32, device="cuda")]
    for x in xs:
        for lanes in (0, 256, 1024):
            c = Z.compress(x, lanes=lanes)
            out = torch.empty_like(x)
            Z.batch_decompress([c], [out], tune=Z.tuning(parts=parts))
            Z.sync_status()
            assert torch.equal(out.view(torch.uint8), x.view(torch.uint8)), (x.dtype, lanes)
            pd = Z.plan_decompress([c], [out], tune=Z.tuning(parts=parts))
            for _ in range(2):
                out.zero_()
                pd.launch()
                Z.sync_status()
                assert torch.equal(out.view(torch.uint8), x.view(torch.uint8)), (x.dtype, lanes)
            pd.close()
    # a mixed-size batch: some chunks split, the ragged ones whole
    cs = [Z.compress(x) for x in xs[:3]]
    outs = [torch.empty_like(x) for x in xs[:3]]
    Z.batch_decompress(cs, outs, tune=Z.tuning(parts=parts))
    Z.sync_status()
    for x, o in zip(xs, outs):
        assert torch.equal(o.view(torch.uint8), x.view(torch.uint8))


@pytest.mark.parametrize("parts,nchunks", [(4, 76), (2, 150), (8, 40)])
def test_cluster_split_with_several_items_per_cta(parts, nchunks):
    """Split launches run as clusters of the chunk's parts that build its table
    together; with one CTA per SM (ctas_per_sm = 1) a cluster takes several
    chunks in turn, and each chunk's table build starts only when every CTA
    of the cluster has finished the previous chunk.  Exact bytes."""
    lanes = 1024 if parts == 8 else 512
    x = W.gaussian(nchunks * 262144 // 2, 0.02, 90 + parts, device="cuda")
    c = Z.compress(x, lanes=lanes)
    out = torch.empty_like(x)
    for tune in (Z.tuning(parts=parts, ctas_per_sm=1), Z.tuning(parts=parts)):
        out.fill_(0)
        Z.batch_decompress([c], [out], tune=tune)
        Z.sync_status()
        assert torch.equal(out.view(torch.int16), x.view(torch.int16))
        pd = Z.plan_decompress([c], [out], tune=tune)
        out.fill_(0)
        pd.launch()
        Z.sync_status()
        pd.close()
        assert torch.equal(out.view(torch.int16), x.view(torch.int16))


def fp32_few_values(n: int, seed: int, random_low_bytes: int) -> torch.Tensor:
    """FP32 values drawn from 37 distinct floats: every byte group has at most
    37 symbols and is Huffman coded; the lowest `random_low_bytes` bytes of
    each element are then replaced by uniform bytes (those groups stay raw)."""
    g = np.random.default_rng(seed)
    vals = g.standard_normal(37).astype(np.float32).view(np.uint32)
    b = vals[g.integers(0, 37, size=n)]
    if random_low_bytes:
        mask = np.uint32((1 << (8 * random_low_bytes)) - 1)
        b = (b & ~mask) | (g.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32) & mask)
    return torch.from_numpy(b.view(np.int32)).view(torch.float32)


@pytest.mark.parametrize("coded", [4, 3, 2])
def test_fp32_chunks_with_several_coded_groups(coded):
    """An FP32 chunk with more than one Huffman group takes the general loop,
    with a table per coded group: the spare tables sit in the stage and the
    raw-word rings behind it, which only the single-coded-group FP32 loop
    uses, so a launch reserves stage + rings (not the stage alone) for three
    of them.  Two, three and four coded groups, three full 256 KiB chunks and
    a ragged one, both CTA sizes and table widths, direct calls and plans,
    alone and in a batch with BF16 and single-coded-group FP32 tensors."""
    x = fp32_few_values(3 * 65536 + 1001, 120 + coded, 4 - coded)
    xs = u8(x)
    c = Z.compress(x.cuda())
    s = c.to_bytes()
    assert s == O.compress(xs, Z.FP32, Z.DEFAULT_CHUNK)
    for ch in range(3):  # the full chunks (the 4 KB tail is too short to code)
        m = _modes(s, ch)
        assert [mode for mode, _ in m] == [1] * coded + [0] * (4 - coded), (ch, m)
    out = torch.empty_like(x, device="cuda")
    for nt in (128, 256):
        for w in (11, 12):
            out.zero_()
            Z.batch_decompress([c], [out], tune=Z.tuning(threads=nt, lut_bits=w))
            Z.sync_status()
            assert np.array_equal(u8(out), xs), (nt, w)
            out.zero_()
            p = Z.plan_decompress([c], [out], tune=Z.tuning(threads=nt, lut_bits=w))
            p.launch()
            Z.sync_status()
            p.close()
            assert np.array_equal(u8(out), xs), ("plan", nt, w)
    ys = [x, W.gaussian(2 * 131072 + 3, 0.02, 124), W.gaussian(65536 + 7, 0.05, 125, torch.float32)]
    cs = [c] + [Z.compress(y.cuda()) for y in ys[1:]]
    outs = [torch.empty_like(y, device="cuda") for y in ys]
    for nt in (128, 256):
        for o in outs:
            o.zero_()
        Z.batch_decompress(cs, outs, tune=Z.tuning(threads=nt))
        Z.sync_status()
        for y, o in zip(ys, outs):
            assert np.array_equal(u8(o), u8(y)), nt
    # FP32 alone, with a single-coded-group tensor first in the batch
    cs2, ys2 = [cs[2], c], [ys[2], x]
    outs2 = [torch.empty_like(y, device="cuda") for y in ys2]
    p = Z.plan_decompress(cs2, outs2)
    p.launch()
    Z.sync_status()
    p.close()
    for y, o in zip(ys2, outs2):
        assert np.array_equal(u8(o), u8(y))
