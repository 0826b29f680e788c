"""Autotuner for the batched codec: chunk size, sub-stream lanes, decode table
width, decoder CTA size and persistent-grid occupancy.

Chunk size (64 KiB - 1 MiB) and lanes are container parameters (chosen at
compression time, recorded in the header); table width W (10-12 bits), threads
per CTA (128 / 256) and CTAs per SM are decoder launch parameters.  None of them changes the decoded bytes.
The tuner compresses a representative sample with each candidate chunk size,
times the graph-captured batched decode for each decoder setting, and keeps
the fastest decode (compression speed breaks ties).  Results are cached as JSON
keyed by (GPU name, dtype, size class) in $ZIPNN_TUNE_CACHE or
~/.cache/zipnn_gb300/tune.json.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import zipnn as Z

CHUNKS = (64 << 10, 128 << 10, 256 << 10, 512 << 10, 1 << 20)
LUT_BITS = (10, 11, 12)


def cache_path() -> str:
    p = os.environ.get("ZIPNN_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "zipnn_gb300", "tune.json")


def size_class(nbytes: int) -> str:
    return f"2^{max(16, int(math.log2(max(1, nbytes))))}"


def key(dtype: int, nbytes: int) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{name}|dtype{dtype}|{size_class(nbytes)}"


def load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def save_cache(d: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = f"{p}.{os.getpid()}.tmp"    # one writer per process (ranks may tune at once)
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _time(fn, reps: int) -> float:
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def tune(sample: list[torch.Tensor], reps: int = 5, chunks=CHUNKS, lut_bits=LUT_BITS,
         ctas=(0, 2, 3, 4), lane_scales=(1, 2), threads=(128, 256),
         verbose: bool = False) -> dict:
    """Sweep the candidates on `sample` (CUDA tensors of one dtype); returns the
    best setting with its measured decode / compress GB/s (original bytes) and,
    under "table", every candidate's figures."""
    orig = sum(t.numel() * t.element_size() for t in sample)
    outs = [torch.empty_like(t) for t in sample]
    results = []
    dtype = Z.dtype_code(sample[0], None)
    # one sub-stream per 1 KiB, or per 512 B, of each chunk (at most 1024)
    cands = sorted({(c, max(1, min(1024, c // 1024 * k, c // 16))) for c in chunks
                    for k in lane_scales})
    for chunk, lanes in cands:
        bc = Z.BatchCompressor(sample, chunk_bytes=chunk, lanes=lanes)
        bc()
        Z.sync_status()
        cs = bc.containers()
        ratio = sum(c.nbytes for c in cs) / orig
        pc = Z.plan_compress(bc)
        t_comp = _time(pc.launch, reps)
        for w, nt, k in [(w, nt, k) for w in lut_bits for nt in threads for k in ctas]:
            if nt != 128 and w < 11:
                continue  # 256-thread CTAs exist for W >= 11 only
            pd = Z.plan_decompress(cs, outs, tune=Z.tuning(threads=nt, ctas_per_sm=k, lut_bits=w))
            t_dec = _time(pd.launch, reps)
            pd.close()
            r = {"chunk_bytes": chunk, "lanes": lanes, "lut_bits": w, "threads": nt,
                 "ctas_per_sm": k, "decode_gbs": orig / t_dec / 1e9,
                 "compress_gbs": orig / t_comp / 1e9, "ratio": ratio}
            results.append(r)
            if verbose:
                print(r, flush=True)
        pc.close()
        del bc, cs
    Z.sync_status()
    best = max(results, key=lambda r: (round(r["decode_gbs"], 0), r["compress_gbs"]))
    best = dict(best)
    best["candidates"] = len(results)
    best["chunks_swept"] = sorted({r["chunk_bytes"] for r in results})
    best["table"] = results
    return best


def tuned(sample: list[torch.Tensor], force: bool = False, nbytes: int | None = None,
          **kw) -> dict:
    """Cached tune() for (GPU, dtype, size class).  The size class is that of
    `nbytes` when given -- the whole workload the sample stands for, so that a
    later lookup for that workload (cached()) finds the setting -- else the
    sample's own size.  The cached entry leaves out the per-candidate table."""
    dtype = Z.dtype_code(sample[0], None)
    if nbytes is None:
        nbytes = sum(t.numel() * t.element_size() for t in sample)
    k = key(dtype, nbytes)
    cache = load_cache()
    if k in cache and not force:
        hit = dict(cache[k])
        hit["from_cache"] = True
        return hit
    best = tune(sample, **kw)
    cache[k] = {kk: v for kk, v in best.items() if kk != "table"}
    try:
        save_cache(cache)
    except OSError:
        pass
    best["from_cache"] = False
    return best


def cached(dtype: int, nbytes: int) -> dict | None:
    """The cached setting for (this GPU, dtype, size class of nbytes), or None.
    The library's Python API consults it when a batched compressor is given no
    chunk size and a decode plan no tuning."""
    return load_cache().get(key(dtype, nbytes))
