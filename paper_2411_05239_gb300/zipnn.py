"""Thin Python binding of libzipnn_gpu.so (argument marshalling only).

Every step of the codec runs in the library's CUDA kernels; this module only
passes device pointers, sizes and the current CUDA stream through the C ABI
declared in ``include/zipnn.h``.  PyTorch provides device memory and streams.
There is no CPU fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libzipnn_gpu.so")

BF16, FP16, FP32, U8 = 0, 1, 2, 3
FLAG_DELTA = 1
DEFAULT_CHUNK = 256 * 1024
TORCH_TO_CODE = {torch.bfloat16: BF16, torch.float16: FP16, torch.float32: FP32,
                 torch.uint8: U8, torch.int8: U8}
CODE_TO_TORCH = {BF16: torch.bfloat16, FP16: torch.float16, FP32: torch.float32, U8: torch.uint8}
ELEM_SIZE = {BF16: 2, FP16: 2, FP32: 4, U8: 1}
STATUS = {0: "ok", -1: "EINVAL", -2: "ENOMEM", -3: "ECORRUPT", -4: "ECUDA", -5: "ETIMEOUT",
          -6: "EBUSY"}

EXPORTS = [
    "zipnn_version", "zipnn_strerror", "zipnn_default_lanes", "zipnn_compress_bound",
    "zipnn_compress_workspace_size", "zipnn_compress", "zipnn_delta", "zipnn_compress_into",
    "zipnn_stream_wrap", "zipnn_decompressed_size", "zipnn_decompress",
    "zipnn_batch_decompress", "zipnn_sync_status", "zipnn_stream_free",
    "zipnn_batch_compress_workspace_size", "zipnn_batch_compress_into",
    "zipnn_plan_decompress", "zipnn_plan_compress", "zipnn_plan_launch", "zipnn_plan_destroy",
    "zipnn_plan_load", "zipnn_batch_compress_into_ex", "zipnn_partition_chunks",
    "zipnn_plan_decompress_range",
]


class ZipnnError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"{what}: {STATUS.get(status, status)} ({status})")
        self.status = status


class ZStream(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("nbytes", ctypes.c_uint64),
                ("orig_nbytes", ctypes.c_uint64), ("dtype", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("chunk_bytes", ctypes.c_uint32),
                ("lanes", ctypes.c_uint32), ("n_chunks", ctypes.c_uint32),
                ("n_groups", ctypes.c_uint32), ("owned", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class ZEncodeOptions(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_uint32), ("probe_skip", ctypes.c_uint32),
                ("encoder", ctypes.c_uint32), ("debug_flags", ctypes.c_uint32)]


class ZTuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("lut_bits", ctypes.c_int32), ("debug_flags", ctypes.c_int32),
                ("parts", ctypes.c_int32)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libzipnn_gpu.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, sz, u32, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_int
    zsp = ctypes.POINTER(ZStream)
    sig = {
        "zipnn_version": ([], i32),
        "zipnn_strerror": ([i32], ctypes.c_char_p),
        "zipnn_default_lanes": ([i32, sz], u32),
        "zipnn_compress_bound": ([sz, i32, sz], sz),
        "zipnn_compress_workspace_size": ([sz, i32, sz], sz),
        "zipnn_compress": ([vp, sz, i32, sz, zsp, vp], i32),
        "zipnn_delta": ([vp, vp, sz, i32, sz, zsp, vp], i32),
        "zipnn_compress_into": ([vp, vp, sz, i32, sz, u32, vp, sz, vp, sz, vp, vp], i32),
        "zipnn_stream_wrap": ([vp, sz, zsp], i32),
        "zipnn_decompressed_size": ([zsp, ctypes.POINTER(sz), ctypes.POINTER(i32)], i32),
        "zipnn_decompress": ([zsp, vp, vp, sz, vp], i32),
        "zipnn_batch_decompress": ([zsp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32,
                                    ctypes.POINTER(ZTuning), vp], i32),
        "zipnn_sync_status": ([vp], i32),
        "zipnn_stream_free": ([zsp], None),
        "zipnn_batch_compress_workspace_size": ([ctypes.POINTER(sz), ctypes.POINTER(i32), i32,
                                                 sz], sz),
        "zipnn_batch_compress_into": ([ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(sz), ctypes.POINTER(i32), i32, sz, u32,
                                       ctypes.POINTER(vp), ctypes.POINTER(sz), vp, sz, vp, vp],
                                      i32),
        "zipnn_plan_decompress": ([zsp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32,
                                   ctypes.POINTER(ZTuning), ctypes.POINTER(vp)], i32),
        "zipnn_plan_compress": ([ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(sz),
                                 ctypes.POINTER(i32), i32, sz, u32, ctypes.POINTER(vp),
                                 ctypes.POINTER(sz), vp, ctypes.POINTER(vp)], i32),
        "zipnn_batch_compress_into_ex": ([ctypes.POINTER(vp), ctypes.POINTER(vp),
                                          ctypes.POINTER(sz), ctypes.POINTER(i32), i32, sz,
                                          ctypes.POINTER(ZEncodeOptions), ctypes.POINTER(vp),
                                          ctypes.POINTER(sz), vp, sz, vp, vp], i32),
        "zipnn_plan_load": ([zsp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                             i32, sz, ctypes.POINTER(ZTuning), ctypes.POINTER(vp)], i32),
        "zipnn_partition_chunks": ([zsp, ctypes.POINTER(vp), i32, i32,
                                    ctypes.POINTER(ctypes.c_uint64)], i32),
        "zipnn_plan_decompress_range": ([zsp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32,
                                         ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.POINTER(ZTuning), ctypes.POINTER(vp)], i32),
        "zipnn_plan_launch": ([vp, vp], i32),
        "zipnn_plan_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ZipnnError(rc, what)


def _sp(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class _CudaView:
    """Expose (pointer, nbytes) of device memory to torch.as_tensor."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "|u1",
                                         "data": (ptr, False), "version": 3}


def device_bytes(ptr: int, n: int) -> torch.Tensor:
    """A uint8 CUDA tensor aliasing n bytes at ptr (no copy)."""
    if n == 0:
        return torch.empty(0, dtype=torch.uint8, device="cuda")
    return torch.as_tensor(_CudaView(ptr, n), device="cuda")


class Compressed:
    """A container in device memory (torch-owned buffer or library-owned)."""

    def __init__(self, zs: ZStream, buffer: torch.Tensor | None = None):
        self.zs = zs
        self.buffer = buffer

    @property
    def nbytes(self) -> int:
        return int(self.zs.nbytes)

    @property
    def orig_nbytes(self) -> int:
        return int(self.zs.orig_nbytes)

    @property
    def dtype_code(self) -> int:
        return int(self.zs.dtype)

    @property
    def is_delta(self) -> bool:
        return bool(self.zs.flags & FLAG_DELTA)

    @property
    def ratio(self) -> float:
        return self.nbytes / max(1, self.orig_nbytes)

    def device_tensor(self) -> torch.Tensor:
        if self.buffer is not None:
            return self.buffer[: self.nbytes]
        return device_bytes(self.zs.data, self.nbytes)

    def to_bytes(self) -> bytes:
        return self.device_tensor().cpu().numpy().tobytes()

    def free(self) -> None:
        if self.zs.owned:
            lib().zipnn_stream_free(ctypes.byref(self.zs))
        self.buffer = None

    def __del__(self):
        try:
            if self.zs.owned:
                lib().zipnn_stream_free(ctypes.byref(self.zs))
        except Exception:
            pass


def _flat_u8(x: torch.Tensor) -> torch.Tensor:
    if not x.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    return x.contiguous().view(-1).view(torch.uint8)


def dtype_code(x: torch.Tensor, dtype: int | None) -> int:
    if dtype is not None:
        return dtype
    if x.dtype not in TORCH_TO_CODE:
        raise ValueError(f"unsupported dtype {x.dtype}")
    return TORCH_TO_CODE[x.dtype]


def default_lanes(dtype: int, chunk_bytes: int) -> int:
    return int(lib().zipnn_default_lanes(dtype, chunk_bytes))


def compress_bound(nbytes: int, dtype: int, chunk_bytes: int) -> int:
    return int(lib().zipnn_compress_bound(nbytes, dtype, chunk_bytes))


def workspace_size(nbytes: int, dtype: int, chunk_bytes: int) -> int:
    return int(lib().zipnn_compress_workspace_size(nbytes, dtype, chunk_bytes))


def compress_into(x: torch.Tensor, out: torch.Tensor, workspace: torch.Tensor,
                  out_nbytes: torch.Tensor | None = None, base: torch.Tensor | None = None,
                  chunk_bytes: int = DEFAULT_CHUNK, lanes: int = 0, dtype: int | None = None,
                  stream=None) -> None:
    """Enqueue compression of x into the caller's buffers (no allocation, no sync)."""
    code = dtype_code(x, dtype)
    src = _flat_u8(x)
    bp = _flat_u8(base).data_ptr() if base is not None else None
    if base is not None and base.numel() * base.element_size() != src.numel():
        raise ValueError("base size differs")
    onp = out_nbytes.data_ptr() if out_nbytes is not None else None
    rc = lib().zipnn_compress_into(src.data_ptr() if src.numel() else None, bp, src.numel(), code,
                                   chunk_bytes, lanes, out.data_ptr(), out.numel(),
                                   workspace.data_ptr(), workspace.numel(), onp, _sp(stream))
    _check(rc, "zipnn_compress_into")


def compress(x: torch.Tensor, chunk_bytes: int = DEFAULT_CHUNK, lanes: int = 0,
             base: torch.Tensor | None = None, dtype: int | None = None, stream=None,
             exact: bool = True) -> Compressed:
    """Compress a CUDA tensor; the container lives in a torch-allocated buffer.
    Reads the container size back (one synchronisation)."""
    code = dtype_code(x, dtype)
    n = x.numel() * x.element_size()
    out = torch.empty(compress_bound(n, code, chunk_bytes), dtype=torch.uint8, device=x.device)
    ws = torch.empty(workspace_size(n, code, chunk_bytes), dtype=torch.uint8, device=x.device)
    onb = torch.zeros(1, dtype=torch.int64, device=x.device)
    compress_into(x, out, ws, onb, base=base, chunk_bytes=chunk_bytes, lanes=lanes, dtype=code,
                  stream=stream)
    total = int(onb.item())
    buf = out[:total].clone() if exact else out
    return wrap(buf, total)


def compress_lib(x: torch.Tensor, chunk_bytes: int = DEFAULT_CHUNK, base: torch.Tensor | None = None,
                 dtype: int | None = None, stream=None) -> Compressed:
    """Compress with the library allocating the container (zipnn_compress / zipnn_delta)."""
    code = dtype_code(x, dtype)
    src = _flat_u8(x)
    zs = ZStream()
    if base is None:
        rc = lib().zipnn_compress(src.data_ptr() if src.numel() else None, src.numel(), code,
                                  chunk_bytes, ctypes.byref(zs), _sp(stream))
        _check(rc, "zipnn_compress")
    else:
        b = _flat_u8(base)
        rc = lib().zipnn_delta(src.data_ptr() if src.numel() else None,
                               b.data_ptr() if b.numel() else None, src.numel(), code,
                               chunk_bytes, ctypes.byref(zs), _sp(stream))
        _check(rc, "zipnn_delta")
    return Compressed(zs, None)


def delta(a: torch.Tensor, b: torch.Tensor, chunk_bytes: int = DEFAULT_CHUNK, lanes: int = 0,
          stream=None) -> Compressed:
    """Container of a XOR b (Sec. 4.2); decode with base=b."""
    return compress(a, chunk_bytes=chunk_bytes, lanes=lanes, base=b, stream=stream)


def wrap(buf: torch.Tensor, nbytes: int | None = None) -> Compressed:
    """Interpret a uint8 CUDA tensor holding a container (reads its header)."""
    if nbytes is None:
        nbytes = buf.numel()
    zs = ZStream()
    rc = lib().zipnn_stream_wrap(buf.data_ptr(), nbytes, ctypes.byref(zs))
    _check(rc, "zipnn_stream_wrap")
    return Compressed(zs, buf)


def decompress(c: Compressed, out: torch.Tensor | None = None, base: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """Decode a container into `out` (allocated if None) on the current stream."""
    if out is None:
        out = torch.empty(c.orig_nbytes // ELEM_SIZE[c.dtype_code],
                          dtype=CODE_TO_TORCH[c.dtype_code], device="cuda")
    o = _flat_u8(out)
    bp = _flat_u8(base).data_ptr() if base is not None else None
    rc = lib().zipnn_decompress(ctypes.byref(c.zs), bp, o.data_ptr() if o.numel() else None,
                                o.numel(), _sp(stream))
    _check(rc, "zipnn_decompress")
    return out


def tuning(threads: int = 0, ctas_per_sm: int = 0, lut_bits: int = 0,
           debug_flags: int = 0, parts: int = 0) -> ZTuning:
    return ZTuning(threads, ctas_per_sm, lut_bits, debug_flags, parts)


def batch_decompress(cs: list[Compressed], outs: list[torch.Tensor],
                     bases: list[torch.Tensor | None] | None = None, tune: ZTuning | None = None,
                     stream=None) -> None:
    """Decode many containers in one persistent launch (device work queue)."""
    n = len(cs)
    arr = (ZStream * n)(*[c.zs for c in cs])
    dsts = (ctypes.c_void_p * n)(*[_flat_u8(o).data_ptr() for o in outs])
    bp = None
    if bases is not None:
        bp = (ctypes.c_void_p * n)(*[(_flat_u8(b).data_ptr() if b is not None else None)
                                     for b in bases])
    rc = lib().zipnn_batch_decompress(arr, bp, dsts, n, ctypes.byref(tune) if tune else None,
                                      _sp(stream))
    _check(rc, "zipnn_batch_decompress")


def sync_status(stream=None) -> None:
    """Wait for the stream and raise if a kernel reported an error."""
    _check(lib().zipnn_sync_status(_sp(stream)), "zipnn_sync_status")


def _ptrs(ts, allow_none=False):
    n = len(ts)
    return (ctypes.c_void_p * n)(*[(_flat_u8(t).data_ptr() if t is not None else None)
                                   for t in ts])


class BatchCompressor:
    """Batched compression of a fixed list of CUDA tensors into caller buffers.

    Arguments are marshalled once; each call() enqueues the four encoder
    kernels for all tensors (zipnn_batch_compress_into_ex).  probe_skip > 0
    applies the skip-ahead probe (Sec. 3.2): after a raw group-chunk the same
    group of the next probe_skip chunks is stored raw.  encoder = 1 selects
    the single-pass encoder where it applies (0: the four kernels)."""

    def __init__(self, xs: list[torch.Tensor], chunk_bytes: int | None = None, lanes: int = 0,
                 bases: list[torch.Tensor | None] | None = None, probe_skip: int = 0,
                 encoder: int = 0, debug_flags: int = 0):
        n = len(xs)
        if chunk_bytes is None:
            # the autotuner's setting for this workload when one is cached,
            # else 256 KiB chunks and the default lanes
            t = tuned_settings(dtype_code(xs[0], None),
                               sum(x.numel() * x.element_size() for x in xs))
            chunk_bytes = int(t["chunk_bytes"]) if t else DEFAULT_CHUNK
            if t and not lanes and bases is None:
                lanes = int(t["lanes"])
        self.xs = xs
        self.chunk_bytes = chunk_bytes
        self.codes = [dtype_code(x, None) for x in xs]
        self.sizes = [x.numel() * x.element_size() for x in xs]
        self.caps = [compress_bound(b, c, chunk_bytes) for b, c in zip(self.sizes, self.codes)]
        dev = xs[0].device
        self.outs = [torch.empty(c, dtype=torch.uint8, device=dev) for c in self.caps]
        self._nb = (ctypes.c_size_t * n)(*self.sizes)
        self._dt = (ctypes.c_int * n)(*self.codes)
        self._caps = (ctypes.c_size_t * n)(*self.caps)
        ws = lib().zipnn_batch_compress_workspace_size(self._nb, self._dt, n, chunk_bytes)
        if ws == 0:
            raise ZipnnError(-1, "zipnn_batch_compress_workspace_size")
        self.ws = torch.empty(ws, dtype=torch.uint8, device=dev)
        self.out_nbytes = torch.zeros(n, dtype=torch.int64, device=dev)
        self._srcs = _ptrs(xs)
        self._bases = _ptrs(bases) if bases is not None else None
        self._outs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in self.outs])
        self.lanes = lanes
        self.opts = ZEncodeOptions(lanes, probe_skip, encoder, debug_flags)
        self.n = n

    def __call__(self, stream=None) -> None:
        rc = lib().zipnn_batch_compress_into_ex(self._srcs, self._bases, self._nb, self._dt,
                                                self.n, self.chunk_bytes, ctypes.byref(self.opts),
                                                self._outs, self._caps, self.ws.data_ptr(),
                                                self.ws.numel(), self.out_nbytes.data_ptr(),
                                                _sp(stream))
        _check(rc, "zipnn_batch_compress_into_ex")

    def containers(self) -> list[Compressed]:
        """Wrap the containers written by the last call (synchronises)."""
        sizes = self.out_nbytes.cpu().tolist()
        return [wrap(o, int(s)) for o, s in zip(self.outs, sizes)]


class Plan:
    """A captured CUDA graph of a batched compression or decompression."""

    def __init__(self, handle: int, keep: list):
        self.handle = handle
        self._keep = keep

    def launch(self, stream=None) -> None:
        _check(lib().zipnn_plan_launch(self.handle, _sp(stream)), "zipnn_plan_launch")

    def close(self) -> None:
        if self.handle:
            lib().zipnn_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tuned_settings(dtype: int, nbytes: int) -> dict | None:
    """The autotuner's cached setting for (this GPU, dtype, size class), or None."""
    from . import autotune
    return autotune.cached(dtype, nbytes)


def plan_decompress(cs: list[Compressed], outs: list[torch.Tensor],
                    bases: list[torch.Tensor | None] | None = None,
                    tune: ZTuning | None = None) -> Plan:
    """Graph-captured persistent decode of all containers.  With no tuning
    given, the autotuner's cached decoder setting for the workload is used
    when there is one (the setting changes speed only, never bytes)."""
    n = len(cs)
    if tune is None and n:
        t = tuned_settings(cs[0].dtype_code, sum(c.orig_nbytes for c in cs))
        if t:
            tune = tuning(threads=int(t["threads"]), ctas_per_sm=int(t["ctas_per_sm"]),
                          lut_bits=int(t["lut_bits"]))
    arr = (ZStream * n)(*[c.zs for c in cs])
    dsts = _ptrs(outs)
    bp = _ptrs(bases) if bases is not None else None
    h = ctypes.c_void_p()
    rc = lib().zipnn_plan_decompress(arr, bp, dsts, n, ctypes.byref(tune) if tune else None,
                                     ctypes.byref(h))
    _check(rc, "zipnn_plan_decompress")
    return Plan(h.value, [cs, outs, bases])


def plan_load(cs: list[Compressed], h_containers: list[torch.Tensor], outs: list[torch.Tensor],
              bases: list[torch.Tensor | None] | None = None, segment_bytes: int = 0,
              tune: ZTuning | None = None) -> Plan:
    """Load plan: every launch copies the containers from pinned host buffers
    (h_containers[i], uint8, c.nbytes bytes) into the device containers cs[i]
    and decodes them into outs, segment by segment, copies and decoding
    overlapped, as one CUDA graph."""
    n = len(cs)
    for c, h in zip(cs, h_containers):
        if h.device.type != "cpu" or not h.is_pinned() or h.numel() * h.element_size() < c.nbytes:
            raise ValueError("plan_load: host containers must be pinned CPU tensors of c.nbytes bytes")
    arr = (ZStream * n)(*[c.zs for c in cs])
    hp = (ctypes.c_void_p * n)(*[hc.data_ptr() for hc in h_containers])
    dsts = _ptrs(outs)
    bp = _ptrs(bases) if bases is not None else None
    h = ctypes.c_void_p()
    rc = lib().zipnn_plan_load(arr, hp, bp, dsts, n, segment_bytes,
                               ctypes.byref(tune) if tune else None, ctypes.byref(h))
    _check(rc, "zipnn_plan_load")
    return Plan(h.value, [cs, h_containers, outs, bases])


def partition_chunks(streams: list[ZStream], host_maps: list, world: int) -> list[int]:
    """Split the chunks of the containers (taken in order) into `world`
    contiguous ranges of near-equal decode traffic (zipnn_partition_chunks).
    host_maps[i]: host bytes (numpy uint8 array, bytes or a CPU tensor) holding
    at least container i's header and map.  Returns world + 1 global chunk
    indices; rank r owns [b[r], b[r+1])."""
    import numpy as np
    n = len(streams)
    arr = (ZStream * n)(*streams)
    keep = [np.ascontiguousarray(np.frombuffer(m, dtype=np.uint8)) if isinstance(m, (bytes, bytearray))
            else (m.contiguous().numpy() if isinstance(m, torch.Tensor) else np.ascontiguousarray(m))
            for m in host_maps]
    maps = (ctypes.c_void_p * n)(*[k.ctypes.data if k.size else None for k in keep])
    out = (ctypes.c_uint64 * (world + 1))()
    _check(lib().zipnn_partition_chunks(arr, maps, n, world, out), "zipnn_partition_chunks")
    return [int(v) for v in out]


def range_extents(streams: list[ZStream], lo: int, hi: int) -> list[tuple[int, int, int] | None]:
    """For the global chunk range [lo, hi): per container, (first chunk, byte
    offset, byte count) of its part of the range, or None when it has none."""
    out, g = [], 0
    for s in streams:
        a = max(lo, g) - g
        b = min(hi, g + s.n_chunks) - g
        g += s.n_chunks
        if a >= b or b <= 0:
            out.append(None)
            continue
        start = a * s.chunk_bytes
        end = min(b * s.chunk_bytes, s.orig_nbytes)
        out.append((a, start, end - start))
    return out


def plan_decompress_range(cs: list[Compressed], outs: list, lo: int, hi: int,
                          bases: list | None = None, tune: ZTuning | None = None) -> Plan:
    """Decode plan for the global chunks [lo, hi) of the containers (a rank's
    share of a sharded decode): outs[i] is a CUDA buffer holding exactly
    container i's part of the range (see range_extents), or None when it has
    none; bases[i] likewise holds the base's bytes of that part."""
    n = len(cs)
    arr = (ZStream * n)(*[c.zs for c in cs])
    dsts = (ctypes.c_void_p * n)(*[(_flat_u8(o).data_ptr() if o is not None else None)
                                   for o in outs])
    bp = None
    if bases is not None:
        bp = (ctypes.c_void_p * n)(*[(_flat_u8(b).data_ptr() if b is not None else None)
                                     for b in bases])
    h = ctypes.c_void_p()
    rc = lib().zipnn_plan_decompress_range(arr, bp, dsts, n, lo, hi,
                                           ctypes.byref(tune) if tune else None, ctypes.byref(h))
    _check(rc, "zipnn_plan_decompress_range")
    return Plan(h.value, [cs, outs, bases])


def plan_compress(bc: BatchCompressor) -> Plan:
    h = ctypes.c_void_p()
    rc = lib().zipnn_plan_compress(bc._srcs, bc._bases, bc._nb, bc._dt, bc.n, bc.chunk_bytes,
                                   bc.lanes, bc._outs, bc._caps, bc.out_nbytes.data_ptr(),
                                   ctypes.byref(h))
    _check(rc, "zipnn_plan_compress")
    return Plan(h.value, [bc])


# ---------------------------------------------------------------------------
# Request server (continuous batching with HBM admission)

OP_COMPRESS, OP_DECOMPRESS = 0, 1


class ZRequest(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("d_input", ctypes.c_void_p), ("input_bytes", ctypes.c_uint64),
                ("container", ZStream), ("d_base", ctypes.c_void_p),
                ("chunk_bytes", ctypes.c_uint64), ("tag", ctypes.c_uint64)]


class ZCompletion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("op", ctypes.c_int32), ("d_output", ctypes.c_void_p),
                ("output_bytes", ctypes.c_uint64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ZServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("max_batch", ctypes.c_uint64),
                ("bytes_processed", ctypes.c_uint64), ("arena_used", ctypes.c_uint64),
                ("inputs_charged", ctypes.c_uint64)]


def _server_lib():
    L = lib()
    if getattr(L, "_server_sigs", False):
        return L
    vp = ctypes.c_void_p
    L.zipnn_server_create.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(vp)]
    L.zipnn_server_create.restype = ctypes.c_int
    L.zipnn_server_submit.argtypes = [vp, ctypes.POINTER(ZRequest), ctypes.POINTER(ctypes.c_uint64)]
    L.zipnn_server_submit.restype = ctypes.c_int
    L.zipnn_server_poll.argtypes = [vp, ctypes.POINTER(ZCompletion), ctypes.c_int]
    L.zipnn_server_poll.restype = ctypes.c_int
    L.zipnn_server_release.argtypes = [vp, ctypes.c_uint64]
    L.zipnn_server_release.restype = ctypes.c_int
    L.zipnn_server_drain.argtypes = [vp, ctypes.c_double]
    L.zipnn_server_drain.restype = ctypes.c_int
    L.zipnn_server_get_stats.argtypes = [vp, ctypes.POINTER(ZServerStats)]
    L.zipnn_server_get_stats.restype = ctypes.c_int
    L.zipnn_server_destroy.argtypes = [vp]
    L.zipnn_server_destroy.restype = None
    L._server_sigs = True
    return L


class Server:
    """Continuous-batching request server on the current CUDA device.

    Inputs (tensors, containers, bases) are caller-owned and must stay alive
    until their request completes; outputs live in the server's arena until
    release()."""

    def __init__(self, budget_bytes: int, slots: int = 4):
        self.L = _server_lib()
        h = ctypes.c_void_p()
        _check(self.L.zipnn_server_create(budget_bytes, slots, ctypes.byref(h)),
               "zipnn_server_create")
        self.h = h.value
        self._keep: dict[int, tuple] = {}

    def submit_compress(self, x: torch.Tensor, base: torch.Tensor | None = None,
                        chunk_bytes: int = 0, tag: int = 0) -> int:
        src = _flat_u8(x)
        r = ZRequest()
        r.op = OP_COMPRESS
        r.dtype = dtype_code(x, None)
        r.d_input = src.data_ptr() if src.numel() else None
        r.input_bytes = src.numel()
        r.d_base = _flat_u8(base).data_ptr() if base is not None else None
        r.chunk_bytes = chunk_bytes
        r.tag = tag
        rid = ctypes.c_uint64()
        _check(self.L.zipnn_server_submit(self.h, ctypes.byref(r), ctypes.byref(rid)),
               "zipnn_server_submit")
        self._keep[rid.value] = (x, base)
        return rid.value

    def submit_decompress(self, c: Compressed, base: torch.Tensor | None = None,
                          tag: int = 0) -> int:
        r = ZRequest()
        r.op = OP_DECOMPRESS
        r.container = c.zs
        r.d_base = _flat_u8(base).data_ptr() if base is not None else None
        r.tag = tag
        rid = ctypes.c_uint64()
        _check(self.L.zipnn_server_submit(self.h, ctypes.byref(r), ctypes.byref(rid)),
               "zipnn_server_submit")
        self._keep[rid.value] = (c, base)
        return rid.value

    def poll(self, max_n: int = 1024) -> list[ZCompletion]:
        arr = (ZCompletion * max_n)()
        n = self.L.zipnn_server_poll(self.h, arr, max_n)
        out = [ZCompletion.from_buffer_copy(arr[i]) for i in range(n)]
        for c in out:
            self._keep.pop(c.id, None)
        return out

    def output(self, c: ZCompletion) -> torch.Tensor:
        """The completion's output bytes as a uint8 CUDA tensor (aliases the arena)."""
        return device_bytes(c.d_output, c.output_bytes)

    def release(self, rid: int) -> None:
        _check(self.L.zipnn_server_release(self.h, rid), "zipnn_server_release")

    def drain(self, timeout_s: float = 60.0) -> None:
        _check(self.L.zipnn_server_drain(self.h, timeout_s), "zipnn_server_drain")

    def stats(self) -> ZServerStats:
        st = ZServerStats()
        _check(self.L.zipnn_server_get_stats(self.h, ctypes.byref(st)), "zipnn_server_get_stats")
        return st

    def close(self) -> None:
        if self.h:
            self.L.zipnn_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
