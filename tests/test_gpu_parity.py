"""GPU path vs the CPU oracle, through the C ABI (needs a GB300).

The bar is bit-exactness: compressed containers byte-identical to the oracle's
(same chunking, modes, code tables, sub-stream offsets and bitstreams), and
decoded bytes identical to the input (lossless, ZipNN Sec. 2.3).  Small cases
span several chunks and a ragged tail; the full-size configurations are checked
on sampled chunks against the oracle and by exact round trips on the device.
"""
from __future__ import annotations

import struct

import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05239_gb300 import workloads as W
from paper_2411_05239_gb300 import zipnn as Z
from tests import spec_decoder

pytestmark = pytest.mark.gpu


def u8(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().view(-1).view(torch.uint8).cpu().numpy()


def _case_tensors():
    g = np.random.default_rng(0)
    return [
        ("bf16_gauss", Z.BF16, W.gaussian(70_001, 0.02, 1)),
        ("fp16_gauss", Z.FP16, W.gaussian(40_003, 0.02, 2, torch.float16)),
        ("fp32_gauss", Z.FP32, W.gaussian(30_001, 0.05, 3, torch.float32)),
        ("fp32_clean", Z.FP32, W.gaussian(30_000, 1.0, 4, torch.bfloat16).float()),
        ("u8_skewed", Z.U8, torch.from_numpy(g.geometric(0.4, size=50_011).clip(0, 255).astype(np.uint8))),
        ("bf16_zero", Z.BF16, torch.zeros(9000, dtype=torch.bfloat16)),
        ("bf16_const", Z.BF16, torch.ones(9000, dtype=torch.bfloat16)),
        ("bf16_random_bits", Z.BF16,
         torch.from_numpy(g.integers(0, 65536, size=20_000).astype(np.int16)).view(torch.bfloat16)),
        ("bf16_two_symbols", Z.BF16,
         torch.where(torch.from_numpy(g.random(33_333) < 0.2), 0.5, 1.0).to(torch.bfloat16)),
    ]


CASES = _case_tensors()
GEOMS = [(4096, 0), (16384, 3), (65536, 0), (262144, 0), (8192, 1)]


@pytest.mark.parametrize("name,dtype,x", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("chunk,lanes", GEOMS, ids=[f"c{c}_l{l}" for c, l in GEOMS])
def test_compress_identical_to_oracle(name, dtype, x, chunk, lanes):
    xs = u8(x)
    want = O.compress(xs, dtype, chunk, lanes or None)
    c = Z.compress(x.cuda(), chunk_bytes=chunk, lanes=lanes, dtype=dtype)
    got = c.to_bytes()
    assert len(got) == len(want)
    assert got == want
    y = Z.decompress(c)
    Z.sync_status()
    assert np.array_equal(u8(y), xs)


@pytest.mark.parametrize("name,dtype,x", CASES, ids=[c[0] for c in CASES])
def test_gpu_decodes_oracle_container(name, dtype, x):
    xs = u8(x)
    s = O.compress(xs, dtype, 16384, 5)
    buf = torch.from_numpy(np.frombuffer(s, dtype=np.uint8).copy()).cuda()
    c = Z.wrap(buf)
    y = Z.decompress(c)
    Z.sync_status()
    assert np.array_equal(u8(y), xs)


@pytest.mark.parametrize("n", [0, 1, 7, 8, 9, 2047, 2048, 2049, 131072, 131073])
def test_sizes_and_ragged_tails(n):
    x = W.gaussian(n, 0.02, 50 + n)
    xs = u8(x)
    for chunk in (4096, 262144):
        want = O.compress(xs, Z.BF16, chunk)
        c = Z.compress(x.cuda(), chunk_bytes=chunk)
        assert c.to_bytes() == want
        y = Z.decompress(c)
        Z.sync_status()
        assert np.array_equal(u8(y), xs)


def test_library_allocated_compress_and_delta():
    x = W.gaussian(100_000, 0.02, 5)
    c = Z.compress_lib(x.cuda(), chunk_bytes=65536)
    assert c.zs.owned == 1
    assert c.to_bytes() == O.compress(u8(x), Z.BF16, 65536)
    y = Z.decompress(c)
    Z.sync_status()
    assert torch.equal(y.cpu().view(torch.int16), x.view(torch.int16))
    c.free()
    nxt, base = W.delta_pair(100_000, seed=6)
    d = Z.compress_lib(nxt.cuda(), chunk_bytes=65536, base=base.cuda())
    assert d.to_bytes() == O.delta(u8(nxt), u8(base), Z.BF16, 65536)


def test_delta_identical_and_reversible():
    nxt, base = W.delta_pair(300_001, seed=3)
    want = O.delta(u8(nxt), u8(base), Z.BF16, 65536)
    c = Z.delta(nxt.cuda(), base.cuda(), chunk_bytes=65536)
    assert c.is_delta
    assert c.to_bytes() == want
    y = Z.decompress(c, base=base.cuda())
    Z.sync_status()
    assert torch.equal(y.cpu().view(torch.int16), nxt.view(torch.int16))
    with pytest.raises(Z.ZipnnError):
        Z.decompress(c)                                  # a delta needs its base
    same = Z.delta(base.cuda(), base.cuda(), chunk_bytes=65536)
    modes = {e[2] for e in spec_decoder.parse(same.to_bytes())["entries"]}
    assert modes == {O.ZERO}


def test_batch_decompress_equals_per_tensor():
    xs = [W.gaussian(n, 0.02, 70 + i) for i, n in enumerate([1, 5000, 131072, 300_000, 77])]
    xs.append(W.gaussian(20_000, 0.05, 80, torch.float32))
    cs = [Z.compress(x.cuda(), chunk_bytes=16384) for x in xs]
    outs = [torch.empty_like(x, device="cuda") for x in xs]
    Z.batch_decompress(cs, outs)
    Z.sync_status()
    for x, o in zip(xs, outs):
        assert torch.equal(o.cpu().view(torch.uint8), x.view(torch.uint8))


def test_batch_with_deltas():
    nxt, base = W.delta_pair(200_000, seed=9)
    plain = W.gaussian(50_000, 0.02, 10)
    cs = [Z.delta(nxt.cuda(), base.cuda(), chunk_bytes=16384), Z.compress(plain.cuda(), chunk_bytes=16384)]
    outs = [torch.empty(200_000, dtype=torch.bfloat16, device="cuda"),
            torch.empty(50_000, dtype=torch.bfloat16, device="cuda")]
    Z.batch_decompress(cs, outs, bases=[base.cuda(), None])
    Z.sync_status()
    assert torch.equal(outs[0].cpu().view(torch.int16), nxt.view(torch.int16))
    assert torch.equal(outs[1].cpu().view(torch.int16), plain.view(torch.int16))


def test_corrupt_map_reports_ecorrupt_and_context_survives():
    x = W.gaussian(50_000, 0.02, 11)
    c = Z.compress(x.cuda(), chunk_bytes=16384)
    buf = c.device_tensor().clone()
    h = spec_decoder.parse(c.to_bytes())
    buf[64 + 12] = 7                                     # invalid mode in the first entry
    bad = Z.wrap(buf)
    Z.decompress(bad)
    with pytest.raises(Z.ZipnnError) as e:
        Z.sync_status()
    assert e.value.status == -3
    # random payload bit flips: decode stays in bounds (OK or ECORRUPT)
    rng = np.random.default_rng(12)
    for _ in range(20):
        b2 = c.device_tensor().clone()
        k = int(rng.integers(h["payload"], c.nbytes))
        b2[k] ^= int(1 << int(rng.integers(0, 8)))
        Z.decompress(Z.wrap(b2))
        try:
            Z.sync_status()
        except Z.ZipnnError as err:
            assert err.status == -3
    # the context still works
    y = Z.decompress(c)
    Z.sync_status()
    assert torch.equal(y.cpu().view(torch.int16), x.view(torch.int16))


def test_bad_header_rejected_on_wrap():
    x = W.gaussian(5000, 0.02, 13)
    c = Z.compress(x.cuda(), chunk_bytes=4096)
    buf = c.device_tensor().clone()
    buf[0] = 0
    with pytest.raises(Z.ZipnnError) as e:
        Z.wrap(buf)
    assert e.value.status == -3
    with pytest.raises(Z.ZipnnError):
        Z.wrap(c.device_tensor().clone()[:-16])          # size mismatch


# ---------------------------------------------------------------------------
# full-size configurations

def _map(c: Z.Compressed):
    t = c.device_tensor()
    hdr = t[:64].cpu().numpy().tobytes()
    nch, = struct.unpack_from("<I", hdr, 28)
    G, = struct.unpack_from("<I", hdr, 24)
    P, = struct.unpack_from("<Q", hdr, 32)
    idx = t[64:P].cpu().numpy().tobytes()
    ent = [struct.unpack_from("<QIBB", idx, 16 * i) for i in range(nch * G)]
    return P, G, ent


def _check_sampled_chunks(c: Z.Compressed, x: torch.Tensor, dtype: int, chunks):
    P, G, ent = _map(c)
    t = c.device_tensor()
    xb = x.contiguous().view(-1).view(torch.uint8)
    C = c.zs.chunk_bytes
    for ch in chunks:
        data = xb[ch * C: (ch + 1) * C].cpu().numpy()
        want = O.compress_chunk(data, dtype, c.zs.lanes)
        for g in range(G):
            off, size, mode, value = ent[ch * G + g]
            assert (mode, value, size) == (want[g][0], want[g][1], len(want[g][2])), (ch, g)
            got = t[P + off: P + off + size].cpu().numpy().tobytes()
            assert got == want[g][2], (ch, g)


def test_plain_bf16_8mib_full_identity():
    x = W.plain_bf16(device="cuda")
    want = O.compress(u8(x), Z.BF16, 262144)
    c = Z.compress(x)
    assert c.to_bytes() == want
    y = Z.decompress(c)
    Z.sync_status()
    assert torch.equal(y, x)
    assert 0.64 < c.ratio < 0.68


def test_rowscaled_fp32_256mib_full_identity():
    x = W.rowscaled_fp32(device="cuda")
    c = Z.compress(x)
    want = O.compress(u8(x), Z.FP32, 262144)
    assert c.to_bytes() == want
    y = Z.decompress(c)
    Z.sync_status()
    assert torch.equal(y.view(torch.int32), x.view(torch.int32))
    assert 0.80 < c.ratio < 0.86


def test_checkpoint_delta_full_size_sampled():
    specs = W.delta_specs()
    n = sum(s.numel for s in specs)
    assert n == 1_713_012_736
    nxt, base = W.delta_pair(n, seed=3, device="cuda")
    c = Z.delta(nxt, base)
    y = Z.decompress(c, base=base)
    Z.sync_status()
    assert torch.equal(y.view(torch.int16), nxt.view(torch.int16))
    d = (nxt.view(torch.int16) ^ base.view(torch.int16)).view(torch.bfloat16)
    rng = np.random.default_rng(3)
    chunks = [0, c.zs.n_chunks - 1] + list(rng.integers(0, c.zs.n_chunks, size=6))
    _check_sampled_chunks(c, d, Z.BF16, chunks)
    del y, d


def test_checkpoint_8b_batched_full_size():
    specs = W.llama8b_specs()
    assert len(specs) == 290
    assert sum(s.numel for s in specs) == 8_030_257_152
    ts = W.checkpoint_bf16(specs, seed=2, device="cuda")
    cs = [Z.compress(t) for t in ts]
    outs = [torch.empty_like(t) for t in ts]
    Z.batch_decompress(cs, outs)
    Z.sync_status()
    for t, o in zip(ts, outs):
        assert torch.equal(t.view(torch.int16), o.view(torch.int16))
    ratio = sum(c.nbytes for c in cs) / sum(t.numel() * 2 for t in ts)
    assert 0.64 < ratio < 0.68
    rng = np.random.default_rng(2)
    for i in [0, 1, 7, 8, 289] + list(rng.integers(0, 290, size=3)):
        c = cs[i]
        chunks = sorted({0, c.zs.n_chunks - 1, int(rng.integers(0, c.zs.n_chunks))})
        _check_sampled_chunks(c, ts[i], Z.BF16, chunks)


def test_batch_compress_and_plans_match_oracle():
    xs = [W.gaussian(n, 0.02, 90 + i) for i, n in enumerate([1, 4097, 131072, 250_001])]
    xs.append(W.gaussian(30_000, 0.05, 95, torch.float32))
    xs.append(W.gaussian(10_000, 0.02, 96, torch.float16))
    xd = [x.cuda() for x in xs]
    bc = Z.BatchCompressor(xd, chunk_bytes=16384)
    bc()
    Z.sync_status()
    cs = bc.containers()
    for x, c in zip(xs, cs):
        assert c.to_bytes() == O.compress(u8(x), Z.dtype_code(x, None), 16384)
    # graph-captured compression writes the same containers
    for o in bc.outs:
        o.zero_()
    pc = Z.plan_compress(bc)
    pc.launch()
    Z.sync_status()
    for x, c in zip(xs, bc.containers()):
        assert c.to_bytes() == O.compress(u8(x), Z.dtype_code(x, None), 16384)
    # graph-captured persistent decode, launched twice
    outs = [torch.empty_like(x) for x in xd]
    pd = Z.plan_decompress(cs, outs, tune=Z.tuning(ctas_per_sm=2))
    for _ in range(2):
        for o in outs:
            o.zero_()
        pd.launch()
        Z.sync_status()
        for x, o in zip(xs, outs):
            assert torch.equal(o.cpu().view(torch.uint8), x.view(torch.uint8))
    pd.close()
    pc.close()


def test_batch_compress_deltas():
    nxt, base = W.delta_pair(120_000, seed=21)
    other = W.gaussian(7000, 0.02, 22)
    bc = Z.BatchCompressor([nxt.cuda(), other.cuda()], chunk_bytes=8192,
                           bases=[base.cuda(), None])
    bc()
    Z.sync_status()
    c0, c1 = bc.containers()
    assert c0.is_delta and not c1.is_delta
    assert c0.to_bytes() == O.delta(u8(nxt), u8(base), Z.BF16, 8192)
    assert c1.to_bytes() == O.compress(u8(other), Z.BF16, 8192)


def test_bounded_wait_gives_up_with_etimeout_and_context_survives():
    """Fault injection without faulting the GPU: the decoder is told to wait for
    bytes that never arrive; its bounded wait must give up (ETIMEOUT), the CTAs
    exit cleanly and the next call works."""
    x = W.gaussian(300_000, 0.02, 60)
    c = Z.compress(x.cuda(), chunk_bytes=65536)
    out = torch.empty_like(x, device="cuda")
    Z.batch_decompress([c], [out], tune=Z.tuning(debug_flags=1))
    with pytest.raises(Z.ZipnnError) as e:
        Z.sync_status()
    assert e.value.status == -5
    Z.batch_decompress([c], [out])
    Z.sync_status()
    assert torch.equal(out.cpu().view(torch.int16), x.view(torch.int16))


@pytest.mark.parametrize("w", [10, 11, 12])
@pytest.mark.parametrize("ctas", [0, 1, 3])
def test_decoder_settings_do_not_change_bytes(w, ctas):
    xs = [W.gaussian(n, 0.02, 61 + i) for i, n in enumerate([100_001, 3000, 262_144])]
    xs.append(W.gaussian(50_000, 1.0, 64, torch.bfloat16).float())     # clean FP32
    cs = [Z.compress(x.cuda(), chunk_bytes=65536) for x in xs]
    outs = [torch.empty_like(x, device="cuda") for x in xs]
    Z.batch_decompress(cs, outs, tune=Z.tuning(lut_bits=w, ctas_per_sm=ctas))
    Z.sync_status()
    for x, o in zip(xs, outs):
        assert torch.equal(o.cpu().view(torch.uint8), x.view(torch.uint8))


@pytest.mark.parametrize("lanes", [256, 300, 512])
def test_two_substreams_per_thread_path(lanes):
    """Chunks with >= 2x as many sub-streams as decoder threads take the
    two-streams-per-thread decode loop; bytes must not change."""
    xs = [W.gaussian(n, 0.02, 70 + i) for i, n in enumerate([300_001, 131_072, 5000])]
    cs = []
    for x in xs:
        c = Z.compress(x.cuda(), chunk_bytes=262144, lanes=lanes)
        assert c.to_bytes() == O.compress(u8(x), Z.BF16, 262144, lanes)
        cs.append(c)
    outs = [torch.empty_like(x, device="cuda") for x in xs]
    for w in (10, 12):
        Z.batch_decompress(cs, outs, tune=Z.tuning(lut_bits=w))
        Z.sync_status()
        for x, o in zip(xs, outs):
            assert torch.equal(o.cpu().view(torch.int16), x.view(torch.int16))
    y = Z.decompress(cs[0])
    Z.sync_status()
    assert torch.equal(y.cpu().view(torch.int16), xs[0].view(torch.int16))


@pytest.mark.parametrize("name", __import__("tests.test_oracle_pins", fromlist=["x"]).GOLDEN_CONTAINERS)
def test_gpu_writes_the_golden_containers(name):
    """The hand-derived containers (tests/golden), including the three that sit
    exactly on the mode decisions (raw threshold, one byte below it, SPARSE /
    HUFF size tie): the GPU encoder must write them byte for byte and decode
    them back."""
    from tests.test_oracle_pins import _load_golden
    f, want = _load_golden(name)
    data = np.frombuffer(bytes.fromhex(f["input"].replace(" ", "")), dtype=np.uint8).copy()
    dtype = int(f["dtype"])
    x = torch.from_numpy(data).cuda()
    c = Z.compress(x, chunk_bytes=int(f["chunk_bytes"]), lanes=int(f["lanes"]), dtype=dtype)
    assert c.to_bytes().hex() == want.hex()
    buf = torch.from_numpy(np.frombuffer(want, dtype=np.uint8).copy()).cuda()
    y = Z.decompress(Z.wrap(buf))
    Z.sync_status()
    assert np.array_equal(u8(y), data)



def _check_map_consistent(c: Z.Compressed):
    """Every map offset is the sum of the 16-B padded payload sizes before it,
    and the header's total is the payload offset plus all of them (the chunk
    map of Sec. 5.1), for the whole container."""
    P, G, ent = _map(c)
    run = 0
    for off, size, mode, value in ent:
        assert off == run
        run += (size + 15) // 16 * 16
    hdr = c.device_tensor()[:64].cpu().numpy().tobytes()
    total, = struct.unpack_from("<Q", hdr, 40)
    assert total == P + run == c.nbytes


def test_checkpoint_8b_timed_compress_plan_full_size():
    """The path the benchmark times, at full size: BatchCompressor + the
    graph-captured compression plan over all 290 tensors in ONE job table, at
    256 KiB chunks and 512 lanes.  Every container's map must be consistent;
    at least 3 chunks per tensor (the first, the last and random ones) of 20
    tensors -- the embedding, both norms of a layer, the head and every kind of
    projection -- must equal the oracle's chunk encoding byte for byte; then the
    graph-captured persistent decode must give back every tensor exactly."""
    specs = W.llama8b_specs()
    ts = W.checkpoint_bf16(specs, seed=2, device="cuda")
    bc = Z.BatchCompressor(ts, chunk_bytes=262144, lanes=512)
    pc = Z.plan_compress(bc)
    for o in bc.outs:
        o.fill_(0xA5)                      # stale bytes cannot pass for output
    pc.launch()
    Z.sync_status()
    cs = bc.containers()
    assert all(c.zs.lanes == 512 and c.zs.chunk_bytes == 262144 for c in cs)
    ratio = sum(c.nbytes for c in cs) / sum(t.numel() * 2 for t in ts)
    assert 0.64 < ratio < 0.68
    rng = np.random.default_rng(22)
    names = [s.name for s in specs]
    pick = [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 145, 146, 149, 150, 200, 283, 286, 287, 288, 289]
    assert names[0] == "embed" and names[8].endswith("norm1") and names[289] == "head"
    for i in range(len(cs)):
        if i in pick or i % 29 == 0:
            _check_map_consistent(cs[i])
    for i in pick:
        c = cs[i]
        n = c.zs.n_chunks
        chunks = sorted({0, n - 1} | {int(v) for v in rng.integers(0, n, size=3)})
        _check_sampled_chunks(c, ts[i], Z.BF16, chunks)
    pc.close()
    outs = [torch.empty_like(t) for t in ts]
    pd = Z.plan_decompress(cs, outs)
    pd.launch()
    Z.sync_status()
    for t, o in zip(ts, outs):
        assert torch.equal(t.view(torch.int16), o.view(torch.int16))
    pd.close()
