"""The packer's pass-A variants against the oracle (needs a GB300).

Chunks of 16-bit elements whose exponent group is Huffman coded and whose
sign + fraction group is stored raw (and FP32 chunks with a coded exponent
group and raw other groups) take one of two specialised encoders:
pair lookups when the code's symbols have distinct residues mod 32, single
lookups otherwise; both stage each unit's bits in a shared-memory slot and
re-encode a unit whose slot overflows.  Every variant must write the oracle's
container byte for byte (ZipNN Sec. 3.1, 3.2, 5.1): here with symbol sets that
clash mod 32, four-symbol runs longer than 32 bits, overflowing slots, exact
zeros, deltas, FP16, FP32, every lane split and several chunk sizes.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05239_gb300 import workloads as W
from paper_2411_05239_gb300 import zipnn as Z

pytestmark = pytest.mark.gpu

N = 600_001  # 16-bit elements: several 256 KiB chunks and a ragged tail


def u8(t: torch.Tensor) -> np.ndarray:
    return t.contiguous().view(-1).view(torch.uint8).cpu().numpy()


def _bf16_from_fields(sign, exp, frac) -> torch.Tensor:
    bits = (sign.astype(np.uint32) << 15) | (exp.astype(np.uint32) << 7) | frac.astype(np.uint32)
    return torch.from_numpy(bits.astype(np.uint16).view(np.int16)).view(torch.bfloat16)


def _exps(x: torch.Tensor) -> np.ndarray:
    return (x.view(torch.int16).numpy().view(np.uint16) >> 7) & 0xFF


def _cases():
    g = np.random.default_rng(77)
    out = {}
    out["gauss"] = (W.gaussian(N, 0.02, 70), None)
    # exponents 100 and 132 share residue 4: the single-lookup encoder
    x = W.gaussian(N, 0.02, 71).view(torch.int16).numpy().view(np.uint16).copy()
    e = ((x >> 7) & 0xFF).astype(np.uint32)
    pick = g.random(N)
    e[pick < 0.01] = 100
    e[(pick >= 0.01) & (pick < 0.02)] = 132
    x = (x & 0x807F) | (e.astype(np.uint16) << 7)
    out["clash"] = (torch.from_numpy(x.view(np.int16)).view(torch.bfloat16), None)
    # one dominant exponent, rare ones from a full residue cycle, runs of
    # eight rare symbols: four-symbol codes longer than 32 bits
    exp = np.full(N, 120, dtype=np.uint32)
    rare = g.random(N) < 0.005
    exp[rare] = g.integers(96, 128, size=int(rare.sum()))
    for start in g.integers(0, N - 8, size=400):
        exp[start:start + 8] = g.integers(96, 128, size=8)
    out["long_quads"] = (_bf16_from_fields(g.integers(0, 2, N), exp, g.integers(0, 128, N)), None)
    # exponents uniform over 32 values: ~5 bits per symbol, slots overflow
    out["overflow"] = (_bf16_from_fields(g.integers(0, 2, N), g.integers(96, 128, N),
                                         g.integers(0, 128, N)), None)
    # exact zeros (symbol 0, residue 0) among Gaussian weights
    z = W.gaussian(N, 0.02, 72)
    z[torch.from_numpy(g.random(N) < 0.01)] = 0
    out["zeros"] = (z, None)
    out["fp16"] = (W.gaussian(N, 0.02, 73, torch.float16), None)
    # a delta whose exponent XOR is coded and whose fraction XOR is raw
    out["delta"] = (W.gaussian(N, 0.02, 74), W.gaussian(N, 0.02, 75))
    # FP32: exponent pairs gathered from two elements, three raw byte groups
    out["fp32"] = (W.gaussian(N // 2, 0.05, 76, torch.float32), None)
    out["fp32_delta"] = (W.gaussian(N // 2, 0.05, 77, torch.float32),
                         W.gaussian(N // 2, 0.05, 78, torch.float32))
    f = W.gaussian(N // 2, 0.05, 79, torch.float32).view(torch.int32).numpy().copy()
    pick = g.random(N // 2)
    f[pick < 0.01] = (f[pick < 0.01] & ~(0xFF << 23)) | (100 << 23)   # exponents 100 and 132
    f[(pick >= 0.01) & (pick < 0.02)] = (f[(pick >= 0.01) & (pick < 0.02)] & ~(0xFF << 23)) | (132 << 23)
    out["fp32_clash"] = (torch.from_numpy(f).view(torch.float32), None)
    return out


CASES = _cases()
GEOMS = [(262144, 512), (262144, 256), (65536, 128), (1048576, 512), (131072, 1024)]


def test_case_labels():
    """The cases reach the variants they are named for."""
    def clash(x, chunk_elems):
        e = _exps(x)
        for c0 in range(0, len(e) - chunk_elems + 1, chunk_elems):
            s = np.unique(e[c0:c0 + chunk_elems])
            if len(np.unique(s & 31)) < len(s):
                return True
        return False
    assert not clash(CASES["gauss"][0], 131072)
    assert clash(CASES["clash"][0], 131072)
    assert not clash(CASES["zeros"][0], 131072)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("chunk,lanes", GEOMS, ids=[f"c{c}_l{l}" for c, l in GEOMS])
def test_pack_variants_match_oracle(name, chunk, lanes):
    x, b = CASES[name]
    dt = Z.dtype_code(x, None)
    if b is None:
        want = O.compress(u8(x), dt, chunk, lanes)
    else:
        want = O.delta(u8(x), u8(b), dt, chunk, lanes)
    xd = x.cuda()
    bd = b.cuda() if b is not None else None
    bc = Z.BatchCompressor([xd], chunk_bytes=chunk, lanes=lanes, bases=[bd])
    for o in bc.outs:
        o.fill_(0x5A)
    bc()
    Z.sync_status()
    got = bc.containers()[0].to_bytes()
    assert len(got) == len(want)
    assert got == want
    y = torch.empty_like(xd)
    Z.batch_decompress([bc.containers()[0]], [y], bases=[bd])
    Z.sync_status()
    assert torch.equal(y.view(torch.int16), xd.view(torch.int16))


def test_single_pass_encoder_takes_the_same_paths():
    """The single-pass encoder shares the packer: same bytes."""
    xs = [CASES[k][0].cuda() for k in ("gauss", "clash", "long_quads", "overflow", "zeros")]
    a = Z.BatchCompressor(xs, chunk_bytes=262144, lanes=512, encoder=1)
    a()
    Z.sync_status()
    for x, c in zip(xs, a.containers()):
        assert c.to_bytes() == O.compress(u8(x.cpu()), Z.BF16, 262144, 512)


def _few_values_fp32(n: int, seed: int) -> np.ndarray:
    g = np.random.default_rng(seed)
    vals = g.standard_normal(29).astype(np.float32).view(np.uint32)
    return vals[g.integers(0, 29, size=n)]


@pytest.mark.parametrize("chunk", [262144, 65536])
def test_delta_packer_stages_two_groups(chunk):
    """Launches that hold deltas take the packer instance that stages two coded
    groups in pass A (and encodes any further coded group, and any unit whose
    slot overflows, from the inputs again).  FP32 deltas of few-valued tensors
    code all four XOR groups, BF16 deltas code both; a batch mixing them with
    plain tensors, against the oracle byte for byte, and decoded back."""
    g = np.random.default_rng(140)
    n32 = 3 * 65536 + 777
    b32 = _few_values_fp32(n32, 141)
    x32 = b32.copy()
    pick = g.random(n32) < 0.3
    x32[pick] = _few_values_fp32(int(pick.sum()), 142)
    base32 = torch.from_numpy(b32.view(np.int32)).view(torch.float32)
    next32 = torch.from_numpy(x32.view(np.int32)).view(torch.float32)
    next16, base16 = W.delta_pair(400_003, seed=143)
    plain = W.gaussian(200_001, 0.02, 144)
    xs = [next32, next16, plain]
    bases = [base32, base16, None]
    bc = Z.BatchCompressor([x.cuda() for x in xs], chunk_bytes=chunk,
                           bases=[b.cuda() if b is not None else None for b in bases])
    for o in bc.outs:
        o.fill_(0x5A)
    bc()
    Z.sync_status()
    cs = bc.containers()
    want = [O.delta(u8(next32), u8(base32), Z.FP32, chunk),
            O.delta(u8(next16), u8(base16), Z.BF16, chunk),
            O.compress(u8(plain), Z.BF16, chunk)]
    modes32 = [m for ch in range(2) for m, _ in
               [tuple(want[0][64 + 16 * (ch * 4 + gg) + 12: 64 + 16 * (ch * 4 + gg) + 14])
                for gg in range(4)]]
    assert modes32.count(1) + modes32.count(4) >= 6  # most FP32 XOR groups coded
    for c, w in zip(cs, want):
        assert c.to_bytes() == w
    outs = [torch.empty_like(x, device="cuda") for x in xs]
    Z.batch_decompress(cs, outs, bases=[b.cuda() if b is not None else None for b in bases])
    Z.sync_status()
    for x, o in zip(xs, outs):
        assert torch.equal(o.cpu().view(torch.uint8), x.view(torch.uint8))
