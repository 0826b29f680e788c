"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h (CPU only: no compute call is made here)."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2411_05239_gb300", "libzipnn_gpu.so")


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(zipnn_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2411_05239_gb300 import build_native
        build_native.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    lib.zipnn_strerror.restype = ctypes.c_char_p
    assert lib.zipnn_strerror(-3) == b"corrupt container"
    assert lib.zipnn_version() == 1
    lib.zipnn_default_lanes.restype = ctypes.c_uint32
    lib.zipnn_default_lanes.argtypes = [ctypes.c_int, ctypes.c_size_t]
    assert lib.zipnn_default_lanes(0, 256 * 1024) == 512
    assert lib.zipnn_default_lanes(1, 256 * 1024) == 512
    assert lib.zipnn_default_lanes(2, 256 * 1024) == 256
    assert lib.zipnn_default_lanes(3, 256 * 1024) == 256
    assert lib.zipnn_default_lanes(0, 4096) == 8
    assert lib.zipnn_default_lanes(0, 1 << 20) == 1024
    lib.zipnn_compress_bound.restype = ctypes.c_size_t
    lib.zipnn_compress_bound.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.c_size_t]
    assert lib.zipnn_compress_bound(1 << 20, 0, 1 << 18) == 64 + 4 * 2 * 16 + (1 << 20) + 4 * 2 * 16


def test_lanes_rule_matches_oracle(lib):
    import oracle as O
    lib.zipnn_default_lanes.restype = ctypes.c_uint32
    lib.zipnn_default_lanes.argtypes = [ctypes.c_int, ctypes.c_size_t]
    for dt in (0, 1, 2, 3):
        for c in (4096, 65536, 262144, 1 << 20, 16 << 20):
            assert lib.zipnn_default_lanes(dt, c) == O.default_lanes(dt, c)
            # deltas: one sub-stream per 1 KiB for every dtype
            assert O.default_lanes(dt, c, delta=True) == max(1, min(1024, c // 1024))


def test_invalid_arguments_rejected_before_any_launch(lib):
    """Host validation returns EINVAL without touching the device."""
    lib.zipnn_compress_into.restype = ctypes.c_int
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    lib.zipnn_compress_into.argtypes = [vp, vp, sz, ctypes.c_int, sz, ctypes.c_uint32, vp, sz, vp,
                                        sz, vp, vp]
    fake = 0x1000
    # odd byte count for BF16
    assert lib.zipnn_compress_into(fake, None, 3, 0, 4096, 0, fake, 1 << 20, fake, 1 << 20, None,
                                   None) == -1
    # chunk not a multiple of 16 / out of range
    assert lib.zipnn_compress_into(fake, None, 64, 0, 4100, 0, fake, 1 << 20, fake, 1 << 20, None,
                                   None) == -1
    assert lib.zipnn_compress_into(fake, None, 64, 0, 2048, 0, fake, 1 << 20, fake, 1 << 20, None,
                                   None) == -1
    # misaligned source
    assert lib.zipnn_compress_into(fake + 2, None, 64, 0, 4096, 0, fake, 1 << 20, fake, 1 << 20,
                                   None, None) == -1
    # unknown dtype
    assert lib.zipnn_compress_into(fake, None, 64, 9, 4096, 0, fake, 1 << 20, fake, 1 << 20, None,
                                   None) == -1
    # output smaller than the bound
    assert lib.zipnn_compress_into(fake, None, 64, 0, 4096, 0, fake, 16, fake, 1 << 20, None,
                                   None) == -2


def test_batch_workspace_query_needs_no_pointers(lib):
    lib.zipnn_batch_compress_workspace_size.restype = ctypes.c_size_t
    lib.zipnn_batch_compress_workspace_size.argtypes = [ctypes.POINTER(ctypes.c_size_t),
                                                       ctypes.POINTER(ctypes.c_int),
                                                       ctypes.c_int, ctypes.c_size_t]
    nb = (ctypes.c_size_t * 3)(2, 8196, 0)
    dt = (ctypes.c_int * 3)(0, 2, 3)
    assert lib.zipnn_batch_compress_workspace_size(nb, dt, 3, 16384) > 0
    bad = (ctypes.c_size_t * 1)(3)
    assert lib.zipnn_batch_compress_workspace_size(bad, (ctypes.c_int * 1)(0), 1, 16384) == 0


def test_load_plan_validates_before_any_device_work(lib):
    """zipnn_plan_load rejects missing pointers and bad container descriptions
    with EINVAL on the host."""
    vp = ctypes.c_void_p
    lib.zipnn_plan_load.restype = ctypes.c_int
    lib.zipnn_plan_load.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_size_t, vp, vp]
    out = vp()
    assert lib.zipnn_plan_load(None, None, None, None, 1, 0, None, ctypes.byref(out)) == -1
    assert lib.zipnn_plan_load(None, None, None, None, 0, 0, None, ctypes.byref(out)) == -1

    class ZStream(ctypes.Structure):
        _fields_ = [("data", vp), ("nbytes", ctypes.c_uint64), ("orig_nbytes", ctypes.c_uint64),
                    ("dtype", ctypes.c_int32), ("flags", ctypes.c_uint32),
                    ("chunk_bytes", ctypes.c_uint32), ("lanes", ctypes.c_uint32),
                    ("n_chunks", ctypes.c_uint32), ("n_groups", ctypes.c_uint32),
                    ("owned", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    zs = ZStream(0x1008, 96, 128, 0, 0, 4096, 2, 1, 2, 0, 0)        # misaligned device data
    hp = (vp * 1)(0x2000)
    dp = (vp * 1)(0x3000)
    assert lib.zipnn_plan_load(ctypes.byref(zs), hp, None, dp, 1, 0, None, ctypes.byref(out)) == -1
    zs = ZStream(0x1000, 96, 128, 0, 0, 4096, 2, 3, 2, 0, 0)        # chunk count inconsistent
    assert lib.zipnn_plan_load(ctypes.byref(zs), hp, None, dp, 1, 0, None, ctypes.byref(out)) == -1
