"""CPU oracle of the ZipNN codec -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper around ``zipnn_oracle.c``: a plain single-threaded C encoder
and decoder of the chunked, byte-grouped Huffman container (ZipNN, Sec. 3.1,
Sec. 3.2, Sec. 4.2, Sec. 5.1).  Only the test-suite, ``__graft_entry__.smoke``
and ``bench.py``'s CPU baseline load it; the product library never does.  It
shares no code with the CUDA path.

The shared object is built with gcc on first use (or by ``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "zipnn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ENOMEM, ECORRUPT = 0, -1, -2, -3
BF16, FP16, FP32, U8 = 0, 1, 2, 3
RAW, HUFF, ZERO, CONST = 0, 1, 2, 3
DTYPE_SIZE = {BF16: 2, FP16: 2, FP32: 4, U8: 1}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, single-threaded C)."""
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp"])
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        sz = ctypes.c_size_t
        L.or_split.argtypes = [ctypes.c_int, ctypes.c_void_p, sz, ctypes.c_void_p]
        L.or_merge.argtypes = [ctypes.c_int, ctypes.c_void_p, sz, ctypes.c_void_p]
        L.or_code_lengths.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.or_canonical_codes.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.or_default_lanes.argtypes = [ctypes.c_int, ctypes.c_uint32]
        L.or_default_lanes.restype = ctypes.c_uint32
        L.or_default_lanes_delta.argtypes = [ctypes.c_int, ctypes.c_uint32]
        L.or_default_lanes_delta.restype = ctypes.c_uint32
        L.or_bound.argtypes = [sz, ctypes.c_int, sz]
        L.or_bound.restype = sz
        L.or_compress.argtypes = [ctypes.c_void_p, sz, ctypes.c_int, sz, ctypes.c_uint32,
                                  ctypes.c_void_p, sz, ctypes.POINTER(sz)]
        L.or_compress_skip.argtypes = [ctypes.c_void_p, sz, ctypes.c_int, sz, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_void_p, sz, ctypes.c_void_p]
        L.or_delta.argtypes = [ctypes.c_void_p, ctypes.c_void_p, sz, ctypes.c_int, sz,
                               ctypes.c_uint32, ctypes.c_void_p, sz, ctypes.POINTER(sz)]
        L.or_decompress.argtypes = [ctypes.c_void_p, sz, ctypes.c_void_p, ctypes.c_void_p, sz]
        L.or_compress_chunk.argtypes = [ctypes.c_void_p, sz, ctypes.c_int, ctypes.c_uint32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, sz]
        L.or_parse_header.argtypes = [ctypes.c_void_p, sz] + [ctypes.c_void_p] * 6
        del u8p
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _as_u8(x) -> np.ndarray:
    a = np.ascontiguousarray(x)
    return a.view(np.uint8).reshape(-1)


def default_lanes(dtype: int, chunk_bytes: int, delta: bool = False) -> int:
    if delta:
        return int(lib().or_default_lanes_delta(dtype, chunk_bytes))
    return int(lib().or_default_lanes(dtype, chunk_bytes))


def split(dtype: int, data) -> np.ndarray:
    """Byte planes [G, n] of the n elements in ``data`` (Sec. 3.1, 3.2)."""
    src = _as_u8(data)
    es = DTYPE_SIZE[dtype]
    n = src.size // es
    planes = np.zeros((es, n), dtype=np.uint8)
    rc = lib().or_split(dtype, _ptr(src), n, _ptr(planes))
    if rc:
        raise OracleError(rc, "split")
    return planes


def merge(dtype: int, planes: np.ndarray) -> np.ndarray:
    planes = np.ascontiguousarray(planes, dtype=np.uint8)
    n = planes.shape[1]
    dst = np.zeros(n * DTYPE_SIZE[dtype], dtype=np.uint8)
    rc = lib().or_merge(dtype, _ptr(planes), n, _ptr(dst))
    if rc:
        raise OracleError(rc, "merge")
    return dst


def code_lengths(hist) -> np.ndarray:
    """Package-merge code lengths (limit 12) for a 256-bin histogram."""
    h = np.ascontiguousarray(hist, dtype=np.uint32)
    assert h.shape == (256,)
    ln = np.zeros(256, dtype=np.uint8)
    lib().or_code_lengths(_ptr(h), _ptr(ln))
    return ln


def canonical_codes(lengths) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, dtype=np.uint8)
    codes = np.zeros(256, dtype=np.uint32)
    lib().or_canonical_codes(_ptr(ln), _ptr(codes))
    return codes


def bound(nbytes: int, dtype: int, chunk_bytes: int) -> int:
    return int(lib().or_bound(nbytes, dtype, chunk_bytes))


def compress(data, dtype: int, chunk_bytes: int = 256 * 1024, lanes: int | None = None,
             skip: int = 0) -> bytes:
    """Container of `data`; skip > 0 applies the skip-ahead probe (Sec. 3.2):
    after a raw group-chunk the same group of the next `skip` chunks is raw."""
    src = _as_u8(data)
    if lanes is None:
        lanes = default_lanes(dtype, chunk_bytes)
    cap = bound(src.size, dtype, chunk_bytes) + 64
    out = np.zeros(cap, dtype=np.uint8)
    n = ctypes.c_size_t(0)
    if skip:
        rc = lib().or_compress_skip(_ptr(src), src.size, dtype, chunk_bytes, lanes, skip,
                                    _ptr(out), cap, ctypes.byref(n))
    else:
        rc = lib().or_compress(_ptr(src), src.size, dtype, chunk_bytes, lanes, _ptr(out), cap,
                               ctypes.byref(n))
    if rc:
        raise OracleError(rc, "compress")
    return out[: n.value].tobytes()


def delta(a, b, dtype: int, chunk_bytes: int = 256 * 1024, lanes: int | None = None) -> bytes:
    sa, sb = _as_u8(a), _as_u8(b)
    if sa.size != sb.size:
        raise OracleError(EINVAL, "delta")
    if lanes is None:
        lanes = default_lanes(dtype, chunk_bytes, delta=True)
    cap = bound(sa.size, dtype, chunk_bytes) + 64
    out = np.zeros(cap, dtype=np.uint8)
    n = ctypes.c_size_t(0)
    rc = lib().or_delta(_ptr(sa), _ptr(sb), sa.size, dtype, chunk_bytes, lanes, _ptr(out), cap,
                        ctypes.byref(n))
    if rc:
        raise OracleError(rc, "delta")
    return out[: n.value].tobytes()


def header(stream: bytes) -> dict:
    s = np.frombuffer(stream, dtype=np.uint8)
    dt = ctypes.c_int32(0)
    fl, cb, ln, nc = (ctypes.c_uint32(0) for _ in range(4))
    nb = ctypes.c_uint64(0)
    rc = lib().or_parse_header(_ptr(s), s.size, ctypes.byref(dt), ctypes.byref(fl),
                               ctypes.byref(nb), ctypes.byref(cb), ctypes.byref(ln),
                               ctypes.byref(nc))
    if rc:
        raise OracleError(rc, "parse_header")
    return dict(dtype=dt.value, flags=fl.value, nbytes=nb.value, chunk_bytes=cb.value,
                lanes=ln.value, n_chunks=nc.value)


def decompress(stream: bytes, base=None) -> np.ndarray:
    s = np.frombuffer(stream, dtype=np.uint8)
    h = header(stream)
    dst = np.zeros(h["nbytes"], dtype=np.uint8)
    bp = None
    if base is not None:
        b = _as_u8(base)
        if b.size != h["nbytes"]:
            raise OracleError(EINVAL, "decompress")
        bp = _ptr(b)
    rc = lib().or_decompress(_ptr(s), s.size, bp, _ptr(dst), dst.size)
    if rc:
        raise OracleError(rc, "decompress")
    return dst


def compress_chunk(chunk, dtype: int, lanes: int):
    """Encode one chunk's bytes; returns [(mode, value, payload_bytes)] per group."""
    src = _as_u8(chunk)
    G = DTYPE_SIZE[dtype]
    stride = src.size // DTYPE_SIZE[dtype] + 1100
    modes = np.zeros(G, dtype=np.int32)
    values = np.zeros(G, dtype=np.int32)
    sizes = np.zeros(G, dtype=np.uint64)
    pay = np.zeros(stride * G, dtype=np.uint8)
    rc = lib().or_compress_chunk(_ptr(src), src.size, dtype, lanes, _ptr(modes), _ptr(values),
                                 _ptr(sizes), _ptr(pay), stride)
    if rc:
        raise OracleError(rc, "compress_chunk")
    return [(int(modes[g]), int(values[g]),
             pay[g * stride: g * stride + int(sizes[g])].tobytes()) for g in range(G)]
