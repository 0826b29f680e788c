"""The no-allocation compression entry point (zipnn_compress_into_static).

It serves callers that cannot allocate device memory when they compress (a
plugin handed device pointers by a framework whose allocator it cannot reach, a
latency-critical loop, a fixed memory budget): it runs the same encoder kernels
as zipnn_compress_into but keeps its scratch in a fixed array inside the
library.  These tests call it through the C ABI, twice in a row with different
inputs (the shared array keeps the previous call's contents), and require its
containers to equal the workspace-based entry point's byte for byte.  This file
is collected last so that a failure here cannot hide another test's result.
"""
from __future__ import annotations

import ctypes

import pytest
import torch

from paper_2411_05239_gb300 import workloads as W
from paper_2411_05239_gb300 import zipnn as Z

pytestmark = pytest.mark.gpu


def _static_fn():
    f = Z.lib().zipnn_compress_into_static
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    f.argtypes = [vp, vp, sz, ctypes.c_int, sz, ctypes.c_uint32, vp, sz, vp, vp]
    f.restype = ctypes.c_int
    return f


def _static(x: torch.Tensor, base: torch.Tensor | None, code: int, chunk: int) -> bytes:
    f = _static_fn()
    n = x.numel() * x.element_size()
    cap = Z.compress_bound(n, code, chunk)
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    onb = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = f(x.data_ptr(), base.data_ptr() if base is not None else None, n, code, chunk, 0,
           out.data_ptr(), cap, onb.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, Z.STATUS.get(rc, rc)
    Z.sync_status()
    return out[: int(onb.item())].cpu().numpy().tobytes()


def _reference(x: torch.Tensor, base: torch.Tensor | None, chunk: int) -> bytes:
    return Z.compress(x, chunk_bytes=chunk, base=base).to_bytes()


def test_static_scratch_matches_workspace_entry_point_twice():
    torch.cuda.set_device(0)
    a = W.gaussian(3_000_001, 0.02, 31, device="cuda")                 # BF16, ragged tail
    b = W.gaussian(1_000_003, 0.05, 32, torch.float32, device="cuda")  # FP32, other sizes
    for x, code, chunk in ((a, Z.BF16, 262144), (b, Z.FP32, 65536)):
        assert _static(x, None, code, chunk) == _reference(x, None, chunk)
    # second round in a row, opposite order, plus a delta
    nxt, base = W.delta_pair(2_000_000, seed=33, device="cuda")
    assert _static(b, None, Z.FP32, 65536) == _reference(b, None, 65536)
    assert _static(nxt, base, Z.BF16, 262144) == _reference(nxt, base, 262144)
    # the container decodes back to the input
    c = Z.wrap(torch.frombuffer(bytearray(_static(a, None, Z.BF16, 262144)),
                                dtype=torch.uint8).cuda())
    y = Z.decompress(c)
    Z.sync_status()
    assert torch.equal(y.view(torch.int16), a.view(torch.int16))


def test_static_scratch_rejects_oversize_input():
    f = _static_fn()
    # 448 MiB of BF16 at 256 KiB chunks = 1,792 chunks x 2 groups = 3,584 pairs > 3,572.
    # The size check comes before any launch, so the tiny buffer is never touched.
    x = torch.empty(16, dtype=torch.uint8, device="cuda")
    rc = f(x.data_ptr(), None, 448 << 20, Z.BF16, 262144, 0, x.data_ptr(), 1 << 40, None,
           torch.cuda.current_stream().cuda_stream)
    assert rc == -2                      # ZIPNN_ENOMEM


def test_static_scratch_limit_is_exact():
    """The documented limit, 3,572 (chunk, byte group) pairs, is the real one:
    U8 input has one group per chunk, so 3,572 chunks of 4 KiB are accepted
    (and give the workspace entry point's bytes) and 3,573 are refused."""
    f = _static_fn()
    chunk = 4096
    g = torch.Generator(device="cuda").manual_seed(34)
    x = (torch.randn(3572 * chunk, device="cuda", generator=g) * 3).round().clamp(-128, 127)
    x = x.to(torch.int8).view(torch.uint8)
    assert _static(x, None, Z.U8, chunk) == _reference(x, None, chunk)
    big = torch.empty(16, dtype=torch.uint8, device="cuda")
    rc = f(big.data_ptr(), None, 3573 * chunk, Z.U8, chunk, 0, big.data_ptr(), 1 << 40, None,
           torch.cuda.current_stream().cuda_stream)
    assert rc == -2                      # ZIPNN_ENOMEM, before any launch
