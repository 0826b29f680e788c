"""Pins of the CPU oracle against facts fixed outside it (CPU only).

Each test ties one oracle function to something other than its own code: the
numeric value of the floats (exponent extraction, ZipNN Sec. 3.1), textbook
Huffman and brute-force / DP optimality (Huffman-only coding, Sec. 3.1), the
RFC 1951 worked example (canonical codes), hand-derived containers
(tests/golden), an independent pure-Python reader of the format, closed forms
(dyadic sources, two symbols, uniform bytes), losslessness (Sec. 2.3) and the
XOR delta's reversibility (Sec. 4.2).
"""
from __future__ import annotations

import heapq
import itertools
import math
import os
import struct

import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05239_gb300 import workloads as W
from tests import spec_decoder

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# split / merge (exponent extraction + byte grouping)

@pytest.mark.parametrize("dtype", [O.BF16, O.FP16])
def test_split_merge_exhaustive_16bit(dtype):
    x = np.arange(65536, dtype=np.uint16)
    planes = O.split(dtype, x)
    # bijective: every (g0, g1) pair occurs exactly once
    key = planes[0].astype(np.int64) * 256 + planes[1]
    assert np.unique(key).size == 65536
    assert np.array_equal(O.merge(dtype, planes), x.view(np.uint8))


def test_bf16_groups_match_numeric_fields():
    """g0 is the biased exponent and g1 = sign | top-7 fraction bits, computed from
    the VALUE of each BF16 number with frexp (no bit formulas)."""
    bits = np.arange(65536, dtype=np.uint32)
    f = (bits << 16).astype(np.uint32).view(np.float32).astype(np.float64)
    planes = O.split(O.BF16, bits.astype(np.uint16))
    finite = np.isfinite(f) & (f != 0)
    mant, ex = np.frexp(np.abs(f[finite]))          # |f| = mant * 2^ex, mant in [0.5, 1)
    normal = ex - 1 + 127 >= 1
    biased = np.where(normal, ex - 1 + 127, 0)
    frac = np.where(normal, (np.abs(f[finite]) / np.exp2(ex - 1.0) - 1.0) * 128,
                    np.abs(f[finite]) / np.exp2(-126.0) * 128)
    assert np.all(frac == np.floor(frac))
    assert np.array_equal(planes[0][finite], biased.astype(np.uint8))
    sign = np.signbit(f[finite]).astype(np.uint8)
    assert np.array_equal(planes[1][finite], (sign << 7) | frac.astype(np.uint8))
    # infinities / NaNs carry the all-ones exponent, zeros the zero exponent
    assert np.all(planes[0][~np.isfinite(f)] == 0xFF)
    assert np.all(planes[0][f == 0] == 0) and np.all((planes[1][f == 0] & 0x7F) == 0)
    # hand patterns: 1.0 and -1.0
    p = O.split(O.BF16, np.array([0x3F80, 0xBF80], dtype=np.uint16))
    assert list(p[0]) == [0x7F, 0x7F] and list(p[1]) == [0x00, 0x80]


def test_fp16_groups_match_numeric_fields():
    bits = np.arange(65536, dtype=np.uint16)
    f = bits.view(np.float16).astype(np.float64)
    planes = O.split(O.FP16, bits)
    ok = np.isfinite(f) & (np.abs(f) >= 2.0 ** -14)
    mant, ex = np.frexp(np.abs(f[ok]))
    e5 = (ex - 1 + 15).astype(np.int64)
    frac10 = ((np.abs(f[ok]) / np.exp2(ex - 1.0) - 1.0) * 1024).astype(np.int64)
    sign = np.signbit(f[ok]).astype(np.int64)
    assert np.array_equal(planes[0][ok], ((e5 << 3) | (frac10 >> 7)).astype(np.uint8))
    assert np.array_equal(planes[1][ok], ((sign << 7) | (frac10 & 0x7F)).astype(np.uint8))


def test_fp32_groups_match_numeric_fields():
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 32, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    special = np.array([0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00001,
                        0x00000001, 0x807FFFFF, 0x3F800000, 0xBF800000], dtype=np.uint32)
    bits = np.concatenate([bits, special])
    planes = O.split(O.FP32, bits)
    assert np.array_equal(O.merge(O.FP32, planes), bits.view(np.uint8))
    f = bits.view(np.float32).astype(np.float64)
    ok = np.isfinite(f) & (np.abs(f) >= 2.0 ** -126)
    mant, ex = np.frexp(np.abs(f[ok]))
    frac23 = ((np.abs(f[ok]) / np.exp2(ex - 1.0) - 1.0) * 2.0 ** 23).astype(np.int64)
    sign = np.signbit(f[ok]).astype(np.int64)
    assert np.array_equal(planes[0][ok], (ex - 1 + 127).astype(np.uint8))
    assert np.array_equal(planes[1][ok], ((sign << 7) | (frac23 >> 16)).astype(np.uint8))
    assert np.array_equal(planes[2][ok], ((frac23 >> 8) & 0xFF).astype(np.uint8))
    assert np.array_equal(planes[3][ok], (frac23 & 0xFF).astype(np.uint8))


# ---------------------------------------------------------------------------
# code lengths (package-merge, limit 12) and canonical codes

def _cost(hist, lengths):
    return int(np.sum(np.asarray(hist, dtype=np.int64) * np.asarray(lengths, dtype=np.int64)))


def _textbook_huffman(weights):
    """Classic Huffman (1952) by repeatedly joining the two lightest trees."""
    heap = [(w, i, [i]) for i, w in enumerate(weights)]
    heapq.heapify(heap)
    depth = [0] * len(weights)
    uid = len(weights)
    while len(heap) > 1:
        w1, _, a = heapq.heappop(heap)
        w2, _, b = heapq.heappop(heap)
        for s in a + b:
            depth[s] += 1
        heapq.heappush(heap, (w1 + w2, uid, a + b))
        uid += 1
    return depth


def _dp_optimal_cost(weights, limit=12):
    """Exact minimum of sum w*l over prefix codes with lengths <= limit.
    Heavier symbols take non-increasing lengths (exchange argument), so a DP
    over sorted weights and the Kraft budget in units of 2^-limit is exact."""
    w = sorted(weights, reverse=True)
    cap = 1 << limit
    inf = np.iinfo(np.int64).max // 4
    dp = np.full((limit + 1, cap + 1), inf, dtype=np.int64)
    for length in range(1, limit + 1):
        dp[length, 1 << (limit - length)] = w[0] * length
    for wi in w[1:]:
        pm = np.minimum.accumulate(dp, axis=0)        # best with previous length <= l
        nd = np.full_like(dp, inf)
        for length in range(1, limit + 1):
            step = 1 << (limit - length)
            nd[length, step:] = pm[length, :cap + 1 - step] + wi * length
        nd[nd >= inf] = inf
        dp = nd
    return int(dp.min())


def _kraft(lengths):
    ln = [int(x) for x in lengths if x]
    return sum(2.0 ** -x for x in ln)


def _random_hists(rng, count):
    out = []
    for _ in range(count):
        nz = int(rng.integers(2, 257))
        syms = rng.choice(256, size=nz, replace=False)
        h = np.zeros(256, dtype=np.uint32)
        kind = rng.integers(0, 3)
        if kind == 0:
            h[syms] = rng.integers(1, 1000, size=nz)
        elif kind == 1:
            h[syms] = np.maximum(1, (rng.geometric(0.3, size=nz) ** 3))
        else:
            h[syms] = np.maximum(1, (1e5 * rng.dirichlet(np.full(nz, 0.2))).astype(np.uint32))
        out.append(h)
    return out


def test_kraft_equality_and_length_limit():
    rng = np.random.default_rng(1)
    for h in _random_hists(rng, 300):
        ln = O.code_lengths(h)
        assert np.all((ln > 0) == (h > 0))
        assert ln.max() <= 12
        assert _kraft(ln) == 1.0            # complete code (exact in binary floating point)


def test_equals_textbook_huffman_when_limit_does_not_bind():
    rng = np.random.default_rng(2)
    checked = 0
    for h in _random_hists(rng, 300):
        nzs = np.nonzero(h)[0]
        depth = _textbook_huffman([int(h[s]) for s in nzs])
        if max(depth) > 12:
            continue
        ln = O.code_lengths(h)
        assert _cost(h, ln) == sum(int(h[s]) * d for s, d in zip(nzs, depth))
        checked += 1
    assert checked > 50


def test_brute_force_optimal_small_alphabets():
    rng = np.random.default_rng(3)
    for n in range(2, 8):
        cand = np.array(list(itertools.product(range(1, n + 1), repeat=n)), dtype=np.int64)
        kraft = np.sum(np.exp2(-cand.astype(np.float64)), axis=1)
        cand = cand[kraft <= 1.0]
        for _ in range(12 if n < 7 else 4):
            w = rng.integers(1, 200, size=n)
            h = np.zeros(256, dtype=np.uint32)
            syms = rng.choice(256, size=n, replace=False)
            h[syms] = w
            best = int(np.min(cand @ w))
            assert _cost(h, O.code_lengths(h)) == best


def test_dp_optimal_when_limit_binds():
    # Fibonacci weights make the unlimited Huffman tree n-1 deep (> 12)
    fib = [1, 1]
    while len(fib) < 24:
        fib.append(fib[-1] + fib[-2])
    cases = [fib, [2 ** k for k in range(20)] + [1], list(range(1, 60)) + [10 ** 6] * 3]
    rng = np.random.default_rng(4)
    cases += [list(np.maximum(1, (1e6 * rng.dirichlet(np.full(200, 0.05))).astype(int)))]
    for weights in cases:
        h = np.zeros(256, dtype=np.uint32)
        h[: len(weights)] = weights
        ln = O.code_lengths(h)
        assert ln.max() <= 12 and _kraft(ln) == 1.0
        assert _cost(h, ln) == _dp_optimal_cost(list(weights))
    assert max(_textbook_huffman(fib)) > 12


def test_entropy_bounds():
    rng = np.random.default_rng(5)
    for h in _random_hists(rng, 200):
        nzs = h[h > 0].astype(np.float64)
        n = nzs.sum()
        H = float(-(nzs / n * np.log2(nzs / n)).sum())
        bits = _cost(h, O.code_lengths(h))
        assert n * H <= bits + 1e-6
        if max(_textbook_huffman(list(nzs))) <= 12:
            assert bits < n * (H + 1)


def test_closed_forms():
    h = np.zeros(256, dtype=np.uint32)
    h[[3, 200]] = [5, 1000]
    assert list(O.code_lengths(h)[[3, 200]]) == [1, 1]
    assert np.all(O.code_lengths(np.full(256, 7, dtype=np.uint32)) == 8)
    # dyadic source: p = 2^-1, 2^-2, ..., 2^-11, 2^-11 -> lengths -log2 p exactly
    h = np.zeros(256, dtype=np.uint32)
    probs_log = list(range(1, 12)) + [11]
    for s, k in enumerate(probs_log):
        h[s * 7] = 2 ** (11 - k)
    ln = O.code_lengths(h)
    assert [int(ln[s * 7]) for s in range(12)] == probs_log
    # equal counts: the smaller symbol takes the shorter code
    h = np.zeros(256, dtype=np.uint32)
    h[[10, 20, 30]] = [4, 4, 4]
    ln = O.code_lengths(h)
    assert int(ln[10]) == 1 and int(ln[20]) == 2 and int(ln[30]) == 2


def test_canonical_codes_rfc1951_example():
    txt = open(os.path.join(GOLDEN, "rfc1951_canonical.txt")).read().splitlines()
    fields = dict(line.split(":", 1) for line in txt if line and not line.startswith("#"))
    lengths = [int(x) for x in fields["lengths"].split()]
    want = fields["codes"].split()
    ln = np.zeros(256, dtype=np.uint8)
    ln[: len(lengths)] = lengths
    codes = O.canonical_codes(ln)
    got = [format(int(codes[i]), f"0{lengths[i]}b") for i in range(len(lengths))]
    assert got == want


def test_canonical_codes_prefix_free():
    rng = np.random.default_rng(6)
    for h in _random_hists(rng, 50):
        ln = O.code_lengths(h)
        codes = O.canonical_codes(ln)
        words = [format(int(codes[s]), f"0{int(ln[s])}b") for s in range(256) if ln[s]]
        words.sort()
        for a, b in zip(words, words[1:]):
            assert not b.startswith(a)


# ---------------------------------------------------------------------------
# container: golden vectors, independent reader, round trips

def _load_golden(name):
    fields, stream = {}, []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split(":", 1)
        if k == "stream":
            stream.append(v.replace(" ", ""))
        else:
            fields[k] = v.strip()
    return fields, bytes.fromhex("".join(stream))


GOLDEN_CONTAINERS = ["bf16_two_symbols.txt", "fp32_four_groups.txt", "u8_sparse_vectors.txt",
                     "u8_raw_at_threshold.txt", "u8_huff_below_threshold.txt",
                     "u8_sparse_huff_tie.txt"]


@pytest.mark.parametrize("name", GOLDEN_CONTAINERS)
def test_golden_containers(name):
    f, want = _load_golden(name)
    data = np.frombuffer(bytes.fromhex(f["input"].replace(" ", "")), dtype=np.uint8)
    got = O.compress(data, int(f["dtype"]), int(f["chunk_bytes"]), int(f["lanes"]))
    assert got.hex() == want.hex()
    assert np.array_equal(O.decompress(want), data)
    assert spec_decoder.decode(want) == data.tobytes()


def _inputs(rng):
    yield O.BF16, W.gaussian(5000, 0.02, 7).view(torch.int16).numpy()
    yield O.FP16, W.gaussian(3001, 0.02, 8, torch.float16).view(torch.int16).numpy()
    yield O.FP32, W.gaussian(2500, 0.05, 9, torch.float32).numpy()
    yield O.U8, rng.integers(0, 7, size=4099).astype(np.uint8)
    yield O.BF16, np.zeros(4096, dtype=np.uint16)                       # all ZERO
    yield O.BF16, np.full(2050, 0x3F80, dtype=np.uint16)                # CONST + ZERO
    yield O.BF16, rng.integers(0, 65536, size=3000).astype(np.uint16)   # RAW
    yield O.FP32, W.gaussian(2049, 1.0, 10, torch.bfloat16).float().numpy()  # clean FP32


def test_independent_reader_round_trip():
    rng = np.random.default_rng(7)
    for dtype, x in _inputs(rng):
        for chunk in (4096, 8192):
            for lanes in (1, 2, 3, 8):
                s = O.compress(x, dtype, chunk, lanes)
                assert spec_decoder.decode(s) == x.tobytes()
                assert np.array_equal(O.decompress(s), x.view(np.uint8))


def test_modes_are_hit():
    rng = np.random.default_rng(8)
    seen = set()
    for dtype, x in _inputs(rng):
        s = O.compress(x, dtype, 4096)
        for e in spec_decoder.parse(s)["entries"]:
            seen.add(e[2])
    assert seen == {O.RAW, O.HUFF, O.ZERO, O.CONST}


@pytest.mark.parametrize("n", [0, 1, 2, 7, 8, 9, 2047, 2048, 2049, 16384, 16391])
def test_round_trip_sizes(n):
    x = W.gaussian(n, 0.02, 100 + n).view(torch.int16).numpy()
    for chunk in (4096, 65536):
        s = O.compress(x, O.BF16, chunk)
        h = O.header(s)
        assert h["nbytes"] == 2 * n and h["n_chunks"] == -(-2 * n // chunk)
        assert np.array_equal(O.decompress(s), x.view(np.uint8))


def test_parameter_validation():
    x = np.zeros(100, dtype=np.uint8)
    with pytest.raises(O.OracleError) as e:
        O.compress(x[:99], O.BF16, 4096)               # odd byte count for a 2-byte type
    assert e.value.code == O.EINVAL
    for chunk in (2048, 4100, (16 << 20) + 16):
        with pytest.raises(O.OracleError):
            O.compress(x, O.BF16, chunk)
    with pytest.raises(O.OracleError):
        O.compress(x, O.BF16, 4096, lanes=257)           # more lanes than 16-B vectors


def test_exponent_group_size_on_gaussian():
    """N(0, 0.02) BF16: the exponent group compresses to about a third, the other
    group stays raw (Sec. 3.1: exponent ~33%, BF16 total ~66.6%)."""
    x = W.plain_bf16(1 << 20, seed=0).view(torch.int16).numpy()
    s = O.compress(x, O.BF16)
    h = spec_decoder.parse(s)
    e0 = sum(e[1] for e in h["entries"][0::2])
    assert all(e[2] == O.RAW for e in h["entries"][1::2])
    assert 0.30 < e0 / (1 << 20) < 0.345
    assert 0.64 < len(s) / x.nbytes < 0.68


# ---------------------------------------------------------------------------
# delta (Sec. 4.2) and metamorphic relations

def test_delta_reversible():
    nxt, base = W.delta_pair(50_000, seed=3)
    a = nxt.view(torch.int16).numpy()
    b = base.view(torch.int16).numpy()
    s = O.delta(a, b, O.BF16, 16384)
    assert O.header(s)["flags"] == 1
    assert np.array_equal(O.decompress(s, base=b), a.view(np.uint8))
    assert spec_decoder.decode(s, base=b.tobytes()) == a.tobytes()
    z = O.delta(a, a, O.BF16, 16384)
    assert all(e[2] == O.ZERO for e in spec_decoder.parse(z)["entries"])
    with pytest.raises(O.OracleError):
        O.decompress(s)                                  # a delta needs its base


def _huff_parts(stream, g):
    h = spec_decoder.parse(stream)
    off, size, mode, _ = h["entries"][g]
    p = stream[h["payload"] + off: h["payload"] + off + size]
    nz = sum(p[:12])
    hh = (12 + nz + 3) // 4 * 4
    return mode, p[:12], p[12:12 + nz], p[hh:]


def test_scaling_by_power_of_two_shifts_exponent_symbols():
    x = W.gaussian(2048, 0.02, 12, torch.float32)
    a = O.compress(x.to(torch.bfloat16).view(torch.int16).numpy(), O.BF16, 4096)
    b = O.compress((x * 8).to(torch.bfloat16).view(torch.int16).numpy(), O.BF16, 4096)
    ma, bits_a, syms_a, rest_a = _huff_parts(a, 0)
    mb, bits_b, syms_b, rest_b = _huff_parts(b, 0)
    assert ma == mb == O.HUFF and bits_a == bits_b and rest_a == rest_b
    assert bytes(s + 3 for s in syms_a) == syms_b


def test_negation_flips_only_the_sign_byte_msb():
    x = W.gaussian(2048, 0.02, 13).view(torch.int16).numpy()
    y = (x.view(np.uint16) ^ 0x8000).astype(np.uint16)
    pa, pb = O.split(O.BF16, x), O.split(O.BF16, y)
    assert np.array_equal(pa[0], pb[0]) and np.array_equal(pa[1] ^ 0x80, pb[1])
    a, b = O.compress(x, O.BF16, 4096), O.compress(y, O.BF16, 4096)
    assert _huff_parts(a, 0) == _huff_parts(b, 0)


def test_corrupt_streams_are_rejected_or_decoded_without_crash():
    x = W.gaussian(8192, 0.02, 14).view(torch.int16).numpy()
    s = bytearray(O.compress(x, O.BF16, 4096))
    with pytest.raises(O.OracleError):
        O.decompress(bytes(s[:-16]))                     # truncated
    bad = bytearray(s)
    bad[0] ^= 1
    with pytest.raises(O.OracleError):
        O.decompress(bytes(bad))                         # magic
    rng = np.random.default_rng(15)
    for _ in range(200):
        t = bytearray(s)
        k = int(rng.integers(0, len(t)))
        t[k] ^= 1 << int(rng.integers(0, 8))
        try:
            O.decompress(bytes(t))
        except O.OracleError as e:
            assert e.code in (O.ECORRUPT, O.EINVAL)


def test_bound_holds():
    rng = np.random.default_rng(16)
    x = rng.integers(0, 256, size=100_000).astype(np.uint8)
    s = O.compress(x, O.U8, 4096)
    assert len(s) <= O.bound(x.size, O.U8, 4096)
    hdr = struct.unpack_from("<4sHBBQ", s, 0)
    assert hdr[0] == b"ZNN1"
