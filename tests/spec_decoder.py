"""A second, pure-Python reader of the container, written from the format
specification alone (test helper; shares nothing with oracle/ or the CUDA path).

It parses the header, the chunk map and every payload, decodes HUFF (and
SPARSE: the same, after a bitmap of the vectors that hold a non-zero symbol)
sub-streams with a dictionary of (length, code) -> symbol built from the
code-length counts, and reassembles elements from their byte groups (ZipNN
Sec. 3.1, Sec. 3.2, Sec. 5.1).  Slow; only for small inputs.
"""
from __future__ import annotations

import struct

import numpy as np

ES = {0: 2, 1: 2, 2: 4, 3: 1}


def parse(stream: bytes) -> dict:
    magic, ver, dtype, flags, nbytes, C, T, G, nch, P, total = struct.unpack_from(
        "<4sHBBQIIIIQQ", stream, 0)
    assert magic == b"ZNN1" and ver == 1
    entries = []
    for i in range(nch * G):
        off, size, mode, value, res = struct.unpack_from("<QIBBH", stream, 64 + 16 * i)
        entries.append((off, size, mode, value))
    return dict(dtype=dtype, flags=flags, nbytes=nbytes, chunk_bytes=C, lanes=T, groups=G,
                chunks=nch, payload=P, total=total, entries=entries)


def _decode_huff(p: bytes, m: int, T: int, V: int, sparse: bool = False) -> bytes:
    counts = list(p[:12])
    nz = sum(counts)
    syms = p[12:12 + nz]
    h = (12 + nz + 3) // 4 * 4
    nv = (m + V - 1) // V
    nonzero = [True] * nv
    if sparse:
        nbw = (nv + 31) // 32
        bm = int.from_bytes(p[h:h + 4 * nbw], "little")
        nonzero = [bool(bm >> v & 1) for v in range(nv)]
        h += 4 * nbw
    starts = [0] + [struct.unpack_from("<I", p, h + 4 * k)[0] for k in range(T - 1)]
    bs = p[h + 4 * (T - 1):]
    # canonical assignment: lengths ascending, symbols in table order
    table = {}
    code, k = 0, 0
    for length in range(1, 13):
        for _ in range(counts[length - 1]):
            table[(length, code)] = syms[k]
            code += 1
            k += 1
        code <<= 1
    bits = "".join(format(struct.unpack_from("<I", bs, 4 * w)[0], "032b")
                   for w in range(len(bs) // 4))
    out = bytearray(m)
    for t in range(T):
        pos = starts[t]
        for v in range(t, nv, T):
            if not nonzero[v]:
                continue                       # all-zero vector: no codes
            for j in range(V):
                i = v * V + j
                if i >= m:
                    break
                c, ln = 0, 0
                while True:
                    c = (c << 1) | int(bits[pos])
                    pos += 1
                    ln += 1
                    if (ln, c) in table:
                        break
                    assert ln < 12, "no code matched"
                out[i] = table[(ln, c)]
    return bytes(out)


def _merge(dtype: int, planes: list[bytes], m: int) -> bytes:
    g = [np.frombuffer(x, dtype=np.uint8).astype(np.uint32) for x in planes]
    if dtype in (0, 1):
        x = ((g[1] >> 7) << 15) | (g[0] << 7) | (g[1] & 0x7F)
        return x.astype("<u2").tobytes()
    if dtype == 2:
        x = ((g[1] >> 7) << 31) | (g[0] << 23) | ((g[1] & 0x7F) << 16) | (g[2] << 8) | g[3]
        return x.astype("<u4").tobytes()
    return g[0].astype(np.uint8).tobytes()


def decode(stream: bytes, base: bytes | None = None) -> bytes:
    h = parse(stream)
    es = ES[h["dtype"]]
    V = 16 // es
    out = bytearray()
    for c in range(h["chunks"]):
        nb = min(h["chunk_bytes"], h["nbytes"] - c * h["chunk_bytes"])
        m = nb // es
        planes = []
        for g in range(h["groups"]):
            off, size, mode, value = h["entries"][c * h["groups"] + g]
            p = stream[h["payload"] + off: h["payload"] + off + size]
            if mode == 0:
                planes.append(bytes(p))
            elif mode == 1:
                planes.append(_decode_huff(p, m, h["lanes"], V))
            elif mode == 2:
                planes.append(bytes(m))
            elif mode == 3:
                planes.append(bytes([value]) * m)
            elif mode == 4:
                planes.append(_decode_huff(p, m, h["lanes"], V, sparse=True))
            else:
                raise ValueError(f"unknown mode {mode}")
        out += _merge(h["dtype"], planes, m)
    if h["flags"] & 1:
        out = bytearray(a ^ b for a, b in zip(out, base))
    return bytes(out)
