#!/usr/bin/env python3
"""Benchmark of the GB300 ZipNN codec hot path; prints ONE JSON line.

Workload (default): a synthetic 8B-class decoder-only checkpoint in BF16
(Llama-3.1-8B shapes, 290 tensors, 8,030,257,152 parameters = 16.06 GB), the
stand-in for the paper's Llama-3.1 measurements (ZipNN Table 2, Table 3).
One step = batched compression of all 290 tensors (histogram, code build, map
scan, bit packing: one CUDA-graph launch) followed by batched persistent
decompression of all of them (one CUDA-graph launch).  `value` is the
decompression throughput in GB/s of ORIGINAL bytes (decode is the path timed
first); compression throughput, ratio and latency percentiles ride along.
Inputs (16 GB) are larger than L2 (129 MB), so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun every rank runs its own checkpoint (weak scaling; no data-path
collective); the timed region is bracketed by a barrier and device syncs and
the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import struct
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "decompress/compress GB/s (original bytes) on 1 GB300, % HBM peak; ratio; p99 ms"
FALLBACK_HBM = 6800.0


def peaks() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world: int, local: int):
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)


def all_max(vals: list[float], world: int) -> list[float]:
    if world == 1:
        return vals
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor(vals, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().tolist()


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def kernel_hash() -> str:
    """Hash of the decoder's sources (decode*.cu, decode_kernels.cuh) and the
    shared internal header."""
    csrc = os.path.join(ROOT, "paper_2411_05239_gb300", "csrc")
    files = sorted(f for f in os.listdir(csrc) if f.startswith("decode")) + ["zipnn_internal.cuh"]
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_from_profile(units: float) -> float | None:
    """DRAM bytes per decode launch from the committed ncu summary, if it was
    taken on the current decoder source (else null)."""
    p = os.path.join(ROOT, "profiles", "decode_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("kernel_sha") != kernel_hash():
            return None
        return float(d["dram_bytes_per_orig_byte"]) * units
    except Exception:
        return None


# ---------------------------------------------------------------------------
def oracle_sample(ts: list[torch.Tensor], chunk: int, sample_bytes: int) -> np.ndarray:
    """Evenly spaced chunks of the checkpoint, concatenated on the host."""
    total_chunks = sum(-(-t.numel() * 2 // chunk) for t in ts)
    want = max(1, sample_bytes // chunk)
    stride = max(1, total_chunks // want)
    pieces, k, got = [], 0, 0
    for t in ts:
        b = t.view(torch.uint8)
        n = -(-b.numel() // chunk)
        for c in range(n):
            if k % stride == 0 and got < want and (c + 1) * chunk <= b.numel():
                pieces.append(b[c * chunk:(c + 1) * chunk].cpu().numpy())
                got += 1
            k += 1
    return np.concatenate(pieces)


def time_oracle(sample: np.ndarray, chunk: int, dtype: int | None = None,
                base: np.ndarray | None = None) -> dict:
    """Oracle compress (or delta against `base`) then decompress of `sample`."""
    import oracle as O
    dtype = O.BF16 if dtype is None else dtype
    t0 = time.perf_counter()
    s = O.compress(sample, dtype, chunk) if base is None else O.delta(sample, base, dtype, chunk)
    t1 = time.perf_counter()
    y = O.decompress(s, base)
    t2 = time.perf_counter()
    assert np.array_equal(y, sample)
    return {"compress_s": t1 - t0, "decompress_s": t2 - t1, "bytes": int(sample.size),
            "ratio": len(s) / sample.size}


def time_oracle_threads(sample: np.ndarray, chunk: int, threads: int) -> dict:
    """The oracle chunk-parallel over host threads: each thread compresses then
    decompresses its own chunk-aligned slice of `sample` (the C calls release
    the GIL).  Wall time of the slowest thread per phase."""
    import concurrent.futures as cf
    import oracle as O
    n = sample.size // chunk
    per = -(-n // threads)
    slices = [sample[i * per * chunk:min(n, (i + 1) * per) * chunk] for i in range(threads)]
    slices = [s for s in slices if s.size]
    with cf.ThreadPoolExecutor(len(slices)) as ex:
        t0 = time.perf_counter()
        conts = list(ex.map(lambda s: O.compress(s, O.BF16, chunk), slices))
        t1 = time.perf_counter()
        outs = list(ex.map(O.decompress, conts))
        t2 = time.perf_counter()
    assert all(np.array_equal(o, s) for o, s in zip(outs, slices))
    nb = sum(s.size for s in slices)
    return {"compress_gbs": nb / (t1 - t0) / 1e9, "decompress_gbs": nb / (t2 - t1) / 1e9,
            "threads": len(slices), "bytes": nb}


# ---------------------------------------------------------------------------
def run_reference(args):
    """The oracle (plain single-threaded C, as it stands) on host cores."""
    world, rank, local = dist_info()
    if rank != 0:
        return 0
    from paper_2411_05239_gb300 import workloads as W
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    specs = W.llama8b_specs()
    if dev == "cuda":
        ts = W.checkpoint_bf16(specs, seed=2, device=dev)
    else:  # draw only the first layers on the host: same recipe, bounded cost
        ts = W.checkpoint_bf16(specs[:12], seed=2, device=dev)
    per_step = args.ref_sample_mb << 20
    sample = oracle_sample(ts, args.chunk, per_step * (args.steps + args.warmup))
    del ts
    steps = []
    n = len(sample) // (args.steps + args.warmup) // args.chunk * args.chunk
    for i in range(args.warmup + args.steps):
        r = time_oracle(sample[i * n:(i + 1) * n], args.chunk)
        if i >= args.warmup:
            steps.append(r)
    dec = sum(r["decompress_s"] for r in steps)
    comp = sum(r["compress_s"] for r in steps)
    nb = sum(r["bytes"] for r in steps)
    value = nb / dec / 1e9
    desc = (f"{args.steps} steps x {n >> 20} MiB: evenly spaced {args.chunk >> 10} KiB chunks of "
            "the 8B BF16 checkpoint, oracle compress + decompress, 1 thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (dec + comp) / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded N(0, 0.02/sqrt(2l+1)) BF16 weights, Llama-3.1-8B shapes)",
        "config": {"workload": "llama8b_bf16_checkpoint", "chunk_bytes": args.chunk,
                   "sample": desc},
        "compress_gbs": nb / comp / 1e9, "ratio": statistics.mean(r["ratio"] for r in steps),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def run_gb300(args):
    from paper_2411_05239_gb300 import workloads as W
    from paper_2411_05239_gb300 import zipnn as Z

    world, rank, local = dist_info()
    dist_init(world, local)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hbm_peak, peak_kind = peaks()
    if args.split:      # whole-tensor comparisons and the load path do not apply to a range
        args.per_tensor, args.e2e_steps = 0, 0

    specs = W.llama8b_specs(n_layers=args.layers, vocab=args.vocab)
    ts = W.checkpoint_bf16(specs, seed=2, device=dev)
    orig = sum(t.numel() * 2 for t in ts)

    # autotuned container (chunk size, lanes) and decoder (table width, CTAs/SM)
    # settings, measured on a sample of the checkpoint (embedding rows + 2 layers)
    tuned = None
    lanes = args.lanes
    if args.autotune:
        # the autotuner sweeps chunk sizes 64 KiB - 1 MiB (container), lanes,
        # table width, CTA size and CTAs per SM (decoder) on a sample and caches
        # the winner for this workload (GPU, dtype, size class); the library's
        # Python API then takes the cached setting itself: the compressor below
        # is given no chunk size and the decode plan no tuning
        from paper_2411_05239_gb300 import autotune as AT
        sample = [ts[0][: 64 * 1024 * 1024]] + ts[1:1 + 2 * 9]
        tuned = AT.tuned(sample, nbytes=orig, force=not args.autotune_cache, reps=3,
                         chunks=AT.CHUNKS, lut_bits=(11, 12), ctas=(0, 2, 3))
        if args.autotune_log and "table" in tuned:
            with open(args.autotune_log, "w") as f:
                json.dump(tuned["table"], f)
        args.chunk = tuned["chunk_bytes"]
        args.lut_bits = tuned["lut_bits"]
        args.threads = tuned["threads"]
        args.ctas_per_sm = tuned["ctas_per_sm"]
        torch.cuda.synchronize()
    # compression plan (batched, graph-captured) and a first pass for the sizes
    if args.autotune:
        bc = Z.BatchCompressor(ts, encoder=args.encoder)  # the cached setting
    else:
        bc = Z.BatchCompressor(ts, chunk_bytes=args.chunk, lanes=lanes, encoder=args.encoder)
    bc()
    Z.sync_status()
    cs = bc.containers()
    args.chunk = cs[0].zs.chunk_bytes
    comp_bytes = sum(c.nbytes for c in cs)
    outs = [torch.empty_like(t) for t in ts]
    tune = None if args.autotune else Z.tuning(threads=args.threads, ctas_per_sm=args.ctas_per_sm,
                                               lut_bits=args.lut_bits)
    # plans capture the four-kernel encoder; the single-pass one (--encoder 1)
    # runs as a direct batched call
    comp_plan = Z.plan_compress(bc) if not args.encoder else None

    def compress(s=None):
        if comp_plan is not None:
            comp_plan.launch(s)
        else:
            bc(s)

    if tune is None:
        # the decode plan below takes the cached setting itself; this copy of it
        # serves the other decoder launches (range plan, load plan)
        tune = Z.tuning(threads=args.threads, ctas_per_sm=args.ctas_per_sm, lut_bits=args.lut_bits)
    split = None
    if args.split:
        # sharded decode of ONE checkpoint (strong scaling): every rank holds the
        # containers of all tensors (compressed identically on every rank) and
        # decodes only its range of chunks, cut from the chunk maps by
        # zipnn_partition_chunks into buffers of just its extents
        zss = [c.zs for c in cs]
        maps = [c.device_tensor()[:64 + 16 * c.zs.n_chunks * c.zs.n_groups].cpu() for c in cs]
        bounds = Z.partition_chunks(zss, maps, world)
        lo, hi = bounds[rank], bounds[rank + 1]
        ext = Z.range_extents(zss, lo, hi)
        outs = [torch.empty(e[2], dtype=torch.uint8, device=dev) if e else None for e in ext]
        dec_plan = Z.plan_decompress_range(cs, outs, lo, hi, tune=tune)
        orig_r = sum(e[2] for e in ext if e)
        comp_r = 0                              # stored payload bytes of the range
        for i, e in enumerate(ext):
            if e is None:
                continue
            G = zss[i].n_groups
            ent = maps[i].numpy().tobytes()
            for ch in range(e[0], e[0] + -(-e[2] // zss[i].chunk_bytes)):
                for g in range(G):
                    size, mode = struct.unpack_from("<IB", ent, 64 + 16 * (ch * G + g) + 8)
                    if mode in (0, 1, 4):       # raw, Huffman, sparse payloads
                        comp_r += (size + 15) // 16 * 16
        split = {"rank_bounds": bounds, "chunks": hi - lo, "orig_bytes": orig_r,
                 "payload_bytes": comp_r}
    elif args.autotune:
        dec_plan = Z.plan_decompress(cs, outs)            # the cached decoder setting
    else:
        dec_plan = Z.plan_decompress(cs, outs, tune=tune)

    # correctness gate before timing (bit-exact round trip on the device)
    compress()
    dec_plan.launch()
    Z.sync_status()
    if split is None:
        for t, o in zip(ts, outs):
            if not torch.equal(t.view(torch.int16), o.view(torch.int16)):
                raise SystemExit("round trip mismatch: refusing to report a number")
    else:
        for t, o, e in zip(ts, outs, ext):
            if e is not None and not torch.equal(t.view(torch.uint8)[e[1]:e[1] + e[2]], o):
                raise SystemExit("range decode mismatch: refusing to report a number")

    stream = torch.cuda.current_stream()
    K, Wm = args.steps, args.warmup
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]

    def step(e=None):
        if e:
            e[0].record(stream)
        compress(stream)
        if e:
            e[1].record(stream)
        dec_plan.launch(stream)
        if e:
            e[2].record(stream)

    for _ in range(Wm):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    t0 = time.perf_counter()
    for k in range(K):
        step(evs[k])
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    Z.sync_status()
    comp_ms = [evs[k][0].elapsed_time(evs[k][1]) for k in range(K)]
    dec_ms = [evs[k][1].elapsed_time(evs[k][2]) for k in range(K)]
    span_ms = evs[0][0].elapsed_time(evs[K - 1][2])
    mc, md, mspan, mwall = all_max([statistics.mean(comp_ms), statistics.mean(dec_ms),
                                    span_ms, wall], world)

    # plain form: one decompress launch per tensor (same buffers)
    pt_ms = None
    if args.per_tensor:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            for c, o in zip(cs, outs):
                Z.decompress(c, out=o)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            for c, o in zip(cs, outs):
                Z.decompress(c, out=o)
        e1.record(stream)
        torch.cuda.synchronize()
        Z.sync_status()
        pt_ms = all_max([e0.elapsed_time(e1) / K], world)[0]

    # end to end through host buffers, every step: the load plan copies the
    # containers from pinned host memory and decodes segment by segment with
    # copies and decoding overlapped (zipnn_plan_load), then the device status
    # word is read back (zipnn_sync_status: 4 bytes D2H).  The round-trip
    # variant also copies every decoded tensor back to pinned host memory.
    e2e = e2e_rt = None
    if args.e2e_steps > 0:
        # one page-locked host buffer per container (page-aligned: copies from
        # 16-B offsets inside one large buffer measured 2-5% slower on this
        # link); the plan copies container by container, segment by segment
        h_cont = [torch.empty(c.nbytes, dtype=torch.uint8, pin_memory=True) for c in cs]
        for h, c in zip(h_cont, cs):
            h.copy_(c.device_tensor())
        torch.cuda.synchronize()
        load = Z.plan_load(cs, h_cont, outs, segment_bytes=args.e2e_segment_mb << 20, tune=tune)

        def e2e_step():
            load.launch(stream)
            Z.sync_status(stream)

        e2e_step()
        for t, o in zip(ts[:3], outs[:3]):
            if not torch.equal(t.view(torch.int16), o.view(torch.int16)):
                raise SystemExit("e2e load mismatch")
        barrier(world)
        torch.cuda.synchronize()
        steps_ms = []
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            e2e_step()
            steps_ms.append((time.perf_counter() - t1) * 1e3)
        torch.cuda.synchronize()
        barrier(world)
        e2e_s = all_max([(time.perf_counter() - t0) / args.e2e_steps], world)[0]
        # the link's pinned H2D rate: one 2 GiB copy (no decode), and the
        # containers' own copies alone
        probe = torch.empty(2 << 30, dtype=torch.uint8, pin_memory=True)
        dprobe = torch.empty(probe.numel(), dtype=torch.uint8, device=dev)
        dconts = [c.device_tensor() for c in cs]
        copy_ms, conts_ms = [], []
        for r in range(4):
            t1 = time.perf_counter()
            dprobe.copy_(probe, non_blocking=True)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            for d, h in zip(dconts, h_cont):
                d.copy_(h, non_blocking=True)
            torch.cuda.synchronize()
            if r:
                copy_ms.append((t2 - t1) * 1e3)
                conts_ms.append((time.perf_counter() - t2) * 1e3)
        h2d_gbs = probe.numel() / (min(copy_ms) / 1e3) / 1e9
        del probe, dprobe, dconts
        # the load's bound: the original bytes that arrive per second when the
        # link carries the containers at that rate
        bound = orig / comp_bytes * h2d_gbs
        steps_ms.sort()
        e2e = {"value": world * orig / e2e_s / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": comp_bytes, "d2h_bytes_per_step": 4,
               "pinned_h2d_gbs": h2d_gbs,
               "copies_alone_ms": min(conts_ms),
               "h2d_bound_gbs": world * bound,
               "frac_of_h2d_bound": orig / e2e_s / 1e9 / bound,
               "frac_of_h2d_bound_median_step": orig / (steps_ms[len(steps_ms) // 2] / 1e3) / 1e9
               / bound,
               "steps": args.e2e_steps, "ms_per_step": e2e_s * 1e3,
               "step_ms_min": steps_ms[0], "step_ms_median": steps_ms[len(steps_ms) // 2],
               "step_ms_max": steps_ms[-1],
               "path": "zipnn_plan_load: pinned host containers -> H2D (copy stream) overlapped "
                       "with per-segment persistent decode into HBM -> zipnn_sync_status (4 B D2H)",
               "segment_mb": args.e2e_segment_mb}
        # round trip: the decoded tensors also go back to pinned host memory
        h_out = [torch.empty(t.numel(), dtype=torch.bfloat16, pin_memory=True) for t in ts]

        def rt_step():
            load.launch(stream)
            for h, o in zip(h_out, outs):
                h.copy_(o, non_blocking=True)
            Z.sync_status(stream)

        rt_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            rt_step()
        torch.cuda.synchronize()
        rt_s = all_max([(time.perf_counter() - t0) / args.e2e_steps], world)[0]
        if not all(torch.equal(h.view(torch.int16), t.view(torch.int16).cpu())
                   for h, t in zip(h_out[:3], ts[:3])):
            raise SystemExit("e2e round trip mismatch")
        e2e_rt = {"value": world * orig / rt_s / 1e9, "unit": "GB/s",
                  "h2d_bytes_per_step": comp_bytes, "d2h_bytes_per_step": orig,
                  "ms_per_step": rt_s * 1e3,
                  "path": "zipnn_plan_load, then every decoded tensor D2H to pinned memory"}
        load.close()
        del h_cont, h_out

    # CPU baseline: the oracle on a bounded sample (rank 0, one GPU only)
    cpu = cpu_n = None
    if rank == 0 and world == 1 and args.cpu_sample_mb > 0:
        sample = oracle_sample(ts, args.chunk, args.cpu_sample_mb << 20)
        r = time_oracle(sample, args.chunk)
        cpu = {"value": r["bytes"] / r["decompress_s"] / 1e9, "unit": "GB/s", "cores": 1,
               "kind": "oracle",
               "compress_gbs": r["bytes"] / r["compress_s"] / 1e9,
               "sample": (f"{r['bytes'] >> 20} MiB: evenly spaced {args.chunk >> 10} KiB chunks "
                          "of the checkpoint; oracle compress then decompress, 1 thread")}
        rn = time_oracle_threads(sample, args.chunk, os.cpu_count() or 1)
        cpu_n = {"value": rn["decompress_gbs"], "unit": "GB/s", "cores": rn["threads"],
                 "kind": "oracle, chunk-parallel over host threads",
                 "compress_gbs": rn["compress_gbs"], "sample": "the same sample, sliced"}

    dec_s, comp_s = md / 1e3, mc / 1e3
    # replicas: every rank decodes its own checkpoint (weak scaling); split: the
    # ranks share one checkpoint, each decoding its range (strong scaling;
    # md is already the slowest rank's time)
    value = (orig if split else world * orig) / dec_s / 1e9
    alg_dec = comp_bytes + orig                 # compressed bytes read + original written
    if split:
        alg_dec = split["payload_bytes"] + split["orig_bytes"]   # this rank's range
    alg_comp = orig + comp_bytes                # original read + compressed written
    traffic = traffic_from_profile(split["orig_bytes"] if split else orig)
    srt = sorted(dec_ms)
    p = lambda q: srt[min(len(srt) - 1, int(math.ceil(q * len(srt))) - 1)]
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": K,
        "warmup": Wm, "ms_per_step": mspan / K, "higher_is_better": True,
        "scaling": "strong" if split else "weak",
        "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded N(0, 0.02/sqrt(2l+1)) BF16 weights, Llama-3.1-8B shapes)",
        "config": {"workload": ("llama8b_bf16_checkpoint" if (args.layers, args.vocab) == (32, 128256)
                                else f"llama_bf16_checkpoint_{args.layers}l_{args.vocab}v"),
                   "tensors": len(ts),
                   "params": orig // 2, "bytes": orig, "chunk_bytes": args.chunk,
                   "lanes": cs[0].zs.lanes, "lut_bits": args.lut_bits or 12, "threads": args.threads or 256,
                   "ctas_per_sm": args.ctas_per_sm,
                   "autotuned": tuned is not None,
                   "autotune": (None if tuned is None else
                                {"chunks_swept": tuned.get("chunks_swept"),
                                 "candidates": tuned.get("candidates"),
                                 "from_cache": tuned.get("from_cache"),
                                 "sample_decode_gbs": tuned.get("decode_gbs")}),
                   "parallelism": (f"split{world}: one checkpoint, chunk ranges per rank"
                                   if split else f"replicas{world}"),
                   "l2": f"inputs ({orig / 1e9:.2f} GB) larger than L2 (129 MB); no flush",
                   "form": ("batched: 1 graph launch compress + 1 graph launch persistent decode"
                            if comp_plan is not None else
                            "batched: 1 single-pass compress call + 1 graph launch persistent "
                            "decode")},
        "split": split,
        "decompress_gbs": value, "compress_gbs": world * orig / comp_s / 1e9,
        "ratio": comp_bytes / orig,
        "decompress_ms": {"mean": md, "p50": p(0.5), "p99": p(0.99)},
        "compress_ms": {"mean": mc},
        "p99_ms": p(0.99),
        "per_tensor_decompress_gbs": (world * orig / (pt_ms / 1e3) / 1e9) if pt_ms else None,
        "roofline": {"kernel": "k_decode (batched persistent decode + merge)", "bound": "hbm",
                     "achieved": alg_dec / dec_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": alg_dec / dec_s / 1e9 / hbm_peak, "peak_kind": peak_kind,
                     "traffic": traffic, "algorithmic_bytes": alg_dec},
        "roofline_compress": {"kernels": "k_hist+k_build+k_scan+k_pack", "bound": "hbm",
                              "achieved": alg_comp / comp_s / 1e9, "peak": hbm_peak,
                              "unit": "GB/s", "frac": alg_comp / comp_s / 1e9 / hbm_peak,
                              "algorithmic_bytes": alg_comp},
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_n,
        "e2e": e2e,
        "e2e_roundtrip": e2e_rt,
        "gpu_launches": 5 * K,
        "clocks": clocks,
        "wall_s_timed": mwall,
        "impl": "gb300",
        "paper_context": "ZipNN CPU: up to 80 GB/s decompression, 13 GB/s compression "
                         "(Xeon Platinum 8480+, 224 cores, 16 workers)",
    }
    # the other the benchmark spec configurations on the same run (rank 0, one GPU):
    # the 3.43 GB checkpoint delta (config 4) and a shortened served stream
    # (config 5: the first requests of the trace, both paths, every result checked)
    if rank == 0 and world == 1 and args.configs:
        del comp_plan, dec_plan, bc, cs, outs, ts
        torch.cuda.empty_cache()
        sub = argparse.Namespace(**vars(args))
        sub.chunk, sub.lanes, sub.threads, sub.lut_bits, sub.ctas_per_sm = 256 << 10, 0, 0, 0, 0
        label, xs, bases = tensor_workload("delta", 24)
        c4 = measure_tensors(label, xs, bases, sub, steps=10, warmup=3, cpu_sample_mb=32)
        del xs, bases
        torch.cuda.empty_cache()
        c5 = measure_serve(sub, args.configs_serve_requests, 200.0)
        torch.cuda.empty_cache()
        line["configs"] = {"c4_checkpoint_delta": c4, "c5_served_stream": c5}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def tensor_workload(name: str, delta_layers: int = 24):
    """(label, tensors, bases) of a single-configuration workload."""
    from paper_2411_05239_gb300 import workloads as W
    bases = None
    if name == "plain":
        xs, label = [W.plain_bf16(device="cuda")], "plain_bf16_8mib"
    elif name == "fp32":
        xs, label = [W.rowscaled_fp32(device="cuda")], "rowscaled_fp32_256mib"
    elif name == "fp16":
        xs = [W.gaussian(134_217_728, 0.02, 9, torch.float16, device="cuda")]
        label = "gaussian_fp16_256mib"
    elif name == "clean_fp32":
        xs, label = [W.clean_fp32_from_bf16(device="cuda")], "clean_fp32_from_bf16_256mib"
    elif name == "clean_fp16":
        xs, label = [W.clean_fp16_from_bf16(device="cuda")], "clean_fp16_from_bf16_128mib"
    else:
        n = sum(sp.numel for sp in W.delta_specs(n_layers=delta_layers))
        nxt, base = W.delta_pair(n, seed=3, device="cuda")
        xs, bases = [nxt], [base]
        label = ("checkpoint_delta_1.7b_bf16" if delta_layers == 24
                 else f"checkpoint_delta_bf16_{delta_layers}l")
    return label, xs, bases


def measure_tensors(label: str, xs, bases, args, steps: int, warmup: int,
                    cpu_sample_mb: int) -> dict:
    """Graph-captured compress + decode of one workload, L2 flushed (256 MB
    write) before each timed phase; CUDA events on the launching stream; the
    oracle on a prefix of the same tensor as the CPU baseline."""
    from paper_2411_05239_gb300 import zipnn as Z
    hbm_peak, peak_kind = peaks()
    orig = sum(x.numel() * x.element_size() for x in xs)
    bc = Z.BatchCompressor(xs, chunk_bytes=args.chunk, bases=bases, lanes=args.lanes,
                           encoder=getattr(args, "encoder", 0))
    bc()
    Z.sync_status()
    cs = bc.containers()
    comp = sum(c.nbytes for c in cs)
    outs = [torch.empty_like(x) for x in xs]
    pc = Z.plan_compress(bc) if not getattr(args, "encoder", 0) else None
    pd = Z.plan_decompress(cs, outs, bases=bases,
                           tune=Z.tuning(threads=args.threads, lut_bits=args.lut_bits,
                                         ctas_per_sm=args.ctas_per_sm,
                                         parts=getattr(args, "parts", 0)))
    pd.launch()
    Z.sync_status()
    for x, o in zip(xs, outs):
        if not torch.equal(x.view(torch.uint8), o.view(torch.uint8)):
            raise SystemExit("round trip mismatch")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    st = torch.cuda.current_stream()
    K = steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    for k in range(warmup + K):
        e = ev[k - warmup] if k >= warmup else None
        flush.fill_(k & 255)
        if e: e[0].record(st)
        if pc is not None:
            pc.launch(st)
        else:
            bc(st)                      # the single-pass encoder: a direct batched call
        if e: e[1].record(st)
        flush.fill_((k + 1) & 255)
        if e: e[2].record(st)
        pd.launch(st)
        if e: e[3].record(st)
    torch.cuda.synchronize()
    Z.sync_status()
    # the timed launches' results are the inputs again
    for x, o in zip(xs, outs):
        if not torch.equal(x.view(torch.uint8), o.view(torch.uint8)):
            raise SystemExit("round trip mismatch after the timed launches")
    cm = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
    dm = sorted(e[2].elapsed_time(e[3]) for e in ev)
    dmean = statistics.mean(dm)
    alg = comp + orig + (orig if bases else 0)
    alg_c = orig + comp + (orig if bases else 0)
    cpu = None
    if cpu_sample_mb > 0:
        lim = max(args.chunk, (cpu_sample_mb << 20) // args.chunk * args.chunk)
        xb = xs[0].view(torch.uint8).reshape(-1)
        samp = xb[:lim].cpu().numpy()
        bsamp = bases[0].view(torch.uint8).reshape(-1)[:lim].cpu().numpy() if bases else None
        r = time_oracle(samp, args.chunk, Z.dtype_code(xs[0], None), bsamp)
        cpu = {"value": r["bytes"] / r["decompress_s"] / 1e9, "unit": "GB/s", "cores": 1,
               "kind": "oracle", "compress_gbs": r["bytes"] / r["compress_s"] / 1e9,
               "sample": f"first {r['bytes'] >> 20} MiB of the tensor"
                         + (" and its base" if bases else "")
                         + "; oracle compress then decompress, 1 thread"}
    if pc is not None:
        pc.close()
    pd.close()
    return {
        "workload": label, "bytes": orig, "chunk_bytes": args.chunk, "steps": K,
        "encoder": "single-pass" if pc is None else "four kernels",
        "decompress_gbs": orig / (dmean / 1e3) / 1e9, "compress_gbs": orig / (cm / 1e3) / 1e9,
        "ratio": comp / orig,
        "decompress_ms": {"mean": dmean, "p99": dm[min(K - 1, int(math.ceil(0.99 * K)) - 1)]},
        "compress_ms": {"mean": cm},
        "roofline": {"kernel": "k_decode", "bound": "hbm", "achieved": alg / (dmean / 1e3) / 1e9,
                     "peak": hbm_peak, "unit": "GB/s",
                     "frac": alg / (dmean / 1e3) / 1e9 / hbm_peak, "peak_kind": peak_kind,
                     "algorithmic_bytes": alg},
        "roofline_compress": {"bound": "hbm", "achieved": alg_c / (cm / 1e3) / 1e9,
                              "peak": hbm_peak, "unit": "GB/s",
                              "frac": alg_c / (cm / 1e3) / 1e9 / hbm_peak},
        "l2": "flushed (256 MB write) before each timed phase",
        "cpu_baseline": cpu,
    }


def run_tensors(args):
    """Single-configuration modes: plain 8 MiB BF16, 256 MiB row-scaled FP32,
    256 MiB N(0, 0.02) FP16, the 3.43 GB checkpoint delta (base + next), and the
    clean-model tensors (FP32 / FP16 holding BF16 values, Sec. 3.2).  Same step
    as the checkpoint mode: graph-captured compress + decode."""
    torch.cuda.set_device(0)
    label, xs, bases = tensor_workload(args.workload, args.delta_layers)
    r = measure_tensors(label, xs, bases, args, args.steps, args.warmup, args.cpu_sample_mb)
    line = {
        "metric": METRIC, "value": r["decompress_gbs"], "unit": "GB/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "u8",
        "data": "synthetic", "config": {"workload": label, "bytes": r["bytes"],
                                        "chunk_bytes": args.chunk, "l2": r["l2"]},
        "compress_gbs": r["compress_gbs"], "ratio": r["ratio"],
        "decompress_ms": r["decompress_ms"], "roofline": r["roofline"],
        "roofline_compress": r["roofline_compress"], "cpu_baseline": r["cpu_baseline"],
        "impl": "gb300",
    }
    print(json.dumps(line), flush=True)
    return 0


class ServeChecks:
    """Checks on a served (or plain) stream's results: every result by device
    identity (a compress result is decoded back on the device and compared
    with its input; a decompress result is compared with its input), and a
    seeded 5% sample of the compress results against the oracle on three
    chunks each (first, last, one random), whose bytes are copied to the host
    at completion and encoded by the oracle after the timed region."""

    def __init__(self, trace, inputs, maxb: int, frac: float = 0.05, seed: int = 4):
        rng = np.random.default_rng(seed)
        self.sample = {r.rid for r in trace if rng.random() < frac}
        self.rng = np.random.default_rng(seed + 1)
        self.inputs = inputs
        self.scratch = torch.empty(maxb + 16, dtype=torch.uint8, device="cuda")
        # comparison result, preallocated: no allocation (which could stall
        # the whole device) while the stream is served
        self.neq = torch.empty(maxb + 16, dtype=torch.bool, device="cuda")
        self.kept = []          # (rid, dtype, lanes, [(chunk bytes, [(mode, value, payload)])])
        self.checked = 0
        # mismatching bytes, summed on the device without waiting for it (the
        # check of a result does not hold up the submitting thread); read once
        # at the end
        self.bad = torch.zeros((), dtype=torch.int64, device="cuda")

    def _stream_of(self, r, out: torch.Tensor):
        """The descriptor of a server-written container, from the request (the
        server compresses at 256 KiB chunks and the default lanes): no header
        read, so no synchronisation."""
        from paper_2411_05239_gb300 import zipnn as Z
        code = {"bf16": Z.BF16, "fp16": Z.FP16, "fp32": Z.FP32}[r.dtype]
        zs = Z.ZStream()
        zs.data = out.data_ptr()
        zs.nbytes = out.numel()
        zs.orig_nbytes = r.nbytes
        zs.dtype = code
        zs.flags = Z.FLAG_DELTA if r.delta else 0
        zs.chunk_bytes = Z.DEFAULT_CHUNK
        zs.lanes = int(Z.lib().zipnn_default_lanes(code, Z.DEFAULT_CHUNK)) if not r.delta \
            else max(1, min(1024, Z.DEFAULT_CHUNK // 1024))
        zs.n_chunks = -(-r.nbytes // Z.DEFAULT_CHUNK)
        zs.n_groups = Z.ELEM_SIZE[code]
        return Z.Compressed(zs, out)

    def check(self, r, out: torch.Tensor) -> None:
        from paper_2411_05239_gb300 import zipnn as Z
        x, b = self.inputs(r)
        xb = x.contiguous().view(-1).view(torch.uint8)
        if r.op == "compress":
            c = self._stream_of(r, out)
            y = self.scratch[:r.nbytes]
            Z.decompress(c, out=y.view(x.dtype) if r.nbytes else y, base=b)
            self._count(y, xb)
            if r.rid in self.sample:
                self.kept.append(self._chunks(r, Z.wrap(out), x, b))
        else:
            self._count(out, xb)
        self.checked += 1

    def _count(self, a: torch.Tensor, b: torch.Tensor) -> None:
        n = a.numel()
        if n != b.numel():
            raise SystemExit("result size differs from the input")
        if n:
            ne = self.neq[:n]
            torch.ne(a, b, out=ne)
            self.bad += ne.sum()

    def reset(self) -> None:
        """Forget the warm-up's checks (kept samples, counts, mismatches)."""
        from paper_2411_05239_gb300 import zipnn as Z
        self.identity_verdict()
        self.kept, self.checked = [], 0
        self.bad.zero_()

    def identity_verdict(self) -> None:
        from paper_2411_05239_gb300 import zipnn as Z
        Z.sync_status()
        if int(self.bad.item()):
            raise SystemExit(f"{int(self.bad.item())} result bytes differ from their inputs")

    def _chunks(self, r, c, x, b):
        import struct
        t = c.device_tensor()
        n, G, C = c.zs.n_chunks, c.zs.n_groups, c.zs.chunk_bytes
        P = 64 + 16 * n * G
        ent = t[64:P].cpu().numpy().tobytes()
        xb = x.contiguous().view(-1).view(torch.uint8)
        if b is not None:
            xb = xb ^ b.contiguous().view(-1).view(torch.uint8)
        out = []
        for ch in sorted({0, n - 1, int(self.rng.integers(0, n))}):
            groups = []
            for g in range(G):
                off, size, mode, value = struct.unpack_from("<QIBB", ent, 16 * (ch * G + g))
                groups.append((mode, value, t[P + off:P + off + size].cpu().numpy().tobytes()))
            out.append((xb[ch * C:(ch + 1) * C].cpu().numpy(), groups))
        return (r.rid, c.dtype_code, c.zs.lanes, out)

    def oracle_verdict(self) -> dict:
        import oracle as O
        self.identity_verdict()
        bad = 0
        for rid, dtype, lanes, chunks in self.kept:
            for data, groups in chunks:
                want = O.compress_chunk(data, dtype, lanes)
                if [(m, v, p) for m, v, p in want] != groups:
                    bad += 1
        if bad:
            raise SystemExit(f"{bad} sampled chunks differ from the oracle")
        return {"identity_checked": self.checked, "oracle_sampled_requests": len(self.kept),
                "oracle_sampled_chunks": sum(len(k[3]) for k in self.kept), "mismatches": 0}


def measure_serve(args, n_requests: int, rate: float) -> dict:
    """Served stream: Poisson arrivals, compress / decompress (70/30),
    BF16/FP16/FP32 (60/20/20), sizes log-uniform in [64 KiB, 2 GiB], 15% deltas
    against a resident base; HBM budget 40 GB.  The served (continuous
    batching) and plain (serial, one stream, one launch per request) paths
    replay the same trace with one clock: latency = completion - SCHEDULED
    arrival (t0 + t_arrival on the host's monotonic clock, the clock the server
    stamps completions with).  After a warm-up, each path replays the trace
    twice: timed, without checks, then untimed with every result checked
    (device identity; a seeded 5% sample of the served compress results also
    against the oracle)."""
    import threading as th
    from paper_2411_05239_gb300 import workloads as W
    from paper_2411_05239_gb300 import zipnn as Z

    torch.cuda.set_device(0)
    trace = W.request_trace(n=n_requests, seed=4, rate=rate)
    maxb = max(r.nbytes for r in trace)
    inputs = W.serve_inputs(trace, device="cuda")
    containers = {}
    for r in trace:
        if r.op == "decompress":
            x, b = inputs(r)
            containers[r.rid] = Z.compress(x, base=b)
    torch.cuda.synchronize()
    checks = ServeChecks(trace, inputs, maxb)

    # warm-up (untimed): a few requests of every kind through a server and the
    # plain calls, so that first launches (kernel loading, pool growth) stay
    # out of both paths' figures
    kinds = {}
    for r in trace:
        kinds.setdefault((r.op, r.dtype, r.delta), r)
    srv = Z.Server(args.serve_budget_gb << 30, slots=args.serve_slots)
    warm_bytes = torch.empty(Z.compress_bound(maxb, Z.FP32, Z.DEFAULT_CHUNK), dtype=torch.uint8,
                             device="cuda")
    warm_ws = torch.empty(Z.workspace_size(maxb, Z.FP32, Z.DEFAULT_CHUNK), dtype=torch.uint8,
                          device="cuda")
    # one of each kind, plain and served one by one, then all of them at once
    # (a burst: batches that mix kinds use their own kernels); the checks'
    # own kernels (decode, compare, sum, XOR) load at first use too
    def finish(want):
        done, t_end = 0, time.monotonic() + 300
        while done < want:
            if time.monotonic() > t_end:
                raise SystemExit("warm-up requests did not complete")
            for c in srv.poll():
                if c.status != 0:
                    raise SystemExit(f"warm-up request {c.tag} failed: {c.status}")
                checks.check(trace[c.tag], srv.output(c))
                torch.cuda.synchronize()
                srv.release(c.id)
                done += 1
            time.sleep(0.001)

    for rnd in range(2):
        for r in kinds.values():
            x, b = inputs(r)
            if r.op == "compress":
                srv.submit_compress(x, base=b, tag=r.rid)
                if rnd == 0:
                    Z.compress_into(x, warm_bytes, warm_ws, base=b)
            else:
                srv.submit_decompress(containers[r.rid], base=b, tag=r.rid)
                if rnd == 0:
                    Z.decompress(containers[r.rid], out=warm_bytes[:r.nbytes].view(x.dtype),
                                 base=b)
            if rnd == 0:
                finish(1)
        if rnd == 1:
            finish(len(kinds))
    srv.close()
    x8 = torch.zeros(64, dtype=torch.uint8, device="cuda")
    (x8 ^ x8).sum().item()
    checks.reset()
    del warm_bytes, warm_ws
    torch.cuda.synchronize()

    def served_replay(check: bool):
        """The trace through a fresh server, arrivals on schedule; with check,
        every result is checked before its output is released."""
        srv = Z.Server(args.serve_budget_gb << 30, slots=args.serve_slots)
        lat, lat_submit, t_span = {}, {}, [None, 0.0]
        t0 = time.monotonic() + 0.5

        def submitter():
            for r in trace:
                dt = t0 + r.t_arrival - time.monotonic()
                if dt > 0:
                    time.sleep(dt)
                x, b = inputs(r)
                if r.op == "compress":
                    srv.submit_compress(x, base=b, tag=r.rid)
                else:
                    srv.submit_decompress(containers[r.rid], base=b, tag=r.rid)
        th_sub = th.Thread(target=submitter)
        switch = sys.getswitchinterval()
        sys.setswitchinterval(5e-5)   # the submitter gets the interpreter back quickly
        th_sub.start()
        held = []   # (server id, event): an output is released once its check has read it
        while len(lat) < len(trace) or held:
            for c in srv.poll():
                if c.status != 0:
                    raise SystemExit(f"served request {c.tag} failed: {c.status}")
                r = trace[c.tag]
                lat[c.tag] = (c.t_done - (t0 + r.t_arrival)) * 1e3
                lat_submit[c.tag] = (c.t_done - c.t_submit) * 1e3
                t_span[0] = (t0 + r.t_arrival if t_span[0] is None
                             else min(t_span[0], t0 + r.t_arrival))
                t_span[1] = max(t_span[1], c.t_done)
                if check:
                    checks.check(r, srv.output(c))
                    ev = torch.cuda.Event()
                    ev.record()
                    held.append((c.id, ev))
                else:
                    srv.release(c.id)
            while held and held[0][1].query():
                srv.release(held.pop(0)[0])
            time.sleep(0.0002)
        th_sub.join()
        sys.setswitchinterval(switch)
        st = srv.stats()
        srv.close()
        return lat, lat_submit, t_span, st

    # the timed served replay carries no checks (they would load the host
    # thread and the GPU in the middle of the measurement); an untimed replay
    # of the same trace checks every result (results do not depend on timing:
    # each is the same alone and in the mix)
    lat, lat_submit, (t_first, t_last), st = served_replay(False)
    done_bytes = sum(r.nbytes for r in trace)
    served = sorted(lat.values())
    served_sub = sorted(lat_submit.values())
    worst = sorted(lat, key=lambda k: -lat[k])[:5]
    worst = [{"rid": k, "op": trace[k].op, "dtype": trace[k].dtype, "delta": trace[k].delta,
              "mb": round(trace[k].nbytes / 2**20, 1), "arrival_s": round(trace[k].t_arrival, 4),
              "ms": round(lat[k], 3), "from_submit_ms": round(lat_submit[k], 3)} for k in worst]
    served_replay(True)

    # plain path: serial, one stream, one launch set per request; timed
    # without checks, then replayed untimed with every result checked
    out_buf = torch.empty(Z.compress_bound(maxb, Z.FP32, Z.DEFAULT_CHUNK), dtype=torch.uint8,
                          device="cuda")   # FP32 has the largest bound and workspace
    ws = torch.empty(Z.workspace_size(maxb, Z.FP32, Z.DEFAULT_CHUNK), dtype=torch.uint8,
                     device="cuda")
    onb = torch.zeros(1, dtype=torch.int64, device="cuda")
    dec_out = torch.empty(maxb // 2 + 16, dtype=torch.int16, device="cuda")
    plain_checks = ServeChecks(trace, inputs, maxb, frac=0.0)

    def plain_replay(check: bool):
        plat = []
        t0 = time.monotonic() + 0.2
        for r in trace:
            dt = t0 + r.t_arrival - time.monotonic()
            if dt > 0 and not check:
                time.sleep(dt)
            x, b = inputs(r)
            if r.op == "compress":
                Z.compress_into(x, out_buf, ws, onb, base=b)
            else:
                c = containers[r.rid]
                Z.decompress(c, out=dec_out.view(torch.uint8)[:c.orig_nbytes].view(x.dtype),
                             base=b)
            torch.cuda.synchronize()
            plat.append((time.monotonic() - (t0 + r.t_arrival)) * 1e3)
            if check:
                if r.op == "compress":
                    plain_checks.check(r, out_buf[:int(onb.item())])
                else:
                    plain_checks.check(r, dec_out.view(torch.uint8)[:r.nbytes])
        return plat

    plain = sorted(plain_replay(False))
    plain_replay(True)
    Z.sync_status()
    verdict = checks.oracle_verdict()
    plain_checks.identity_verdict()
    verdict["plain_identity_checked"] = plain_checks.checked
    verdict["how"] = ("an untimed replay of the trace through the server and one through the "
                      "plain calls, every result checked; the timed replays carry no checks")
    pct = lambda a, q: a[min(len(a) - 1, int(math.ceil(q * len(a))) - 1)]
    total = sum(r.nbytes for r in trace)
    return {
        "workload": "served_stream", "requests": len(trace), "rate_per_s": rate,
        "budget_gb": args.serve_budget_gb, "slots": args.serve_slots, "offered_gb": total / 1e9,
        "latency_origin": "scheduled arrival (t0 + t_arrival), host monotonic clock, both paths",
        "served": {"p50_ms": pct(served, 0.5), "p99_ms": pct(served, 0.99),
                   "mean_ms": statistics.mean(served), "batches": st.batches,
                   "max_batch": st.max_batch, "gbs": done_bytes / (t_last - t_first) / 1e9,
                   "from_submit_p50_ms": pct(served_sub, 0.5),
                   "from_submit_p99_ms": pct(served_sub, 0.99), "slowest": worst},
        "plain": {"p50_ms": pct(plain, 0.5), "p99_ms": pct(plain, 0.99),
                  "mean_ms": statistics.mean(plain)},
        "checks": verdict,
    }


def run_serve(args):
    """Config 5 alone (see measure_serve)."""
    r = measure_serve(args, args.serve_requests, args.serve_rate)
    line = {
        "metric": METRIC, "value": r["served"]["gbs"], "unit": "GB/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "u8", "data": "synthetic",
        "config": {k: r[k] for k in ("workload", "requests", "rate_per_s", "budget_gb", "slots",
                                     "offered_gb", "latency_origin")},
        "served": r["served"], "plain": r["plain"], "checks": r["checks"], "impl": "gb300",
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--chunk", type=int, default=256 * 1024)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--lut-bits", type=int, default=0)
    ap.add_argument("--lanes", type=int, default=0, help="sub-streams per chunk (0 = default)")
    ap.add_argument("--parts", type=int, default=0,
                    help="decoder work items per chunk for the single-tensor workloads "
                         "(0 = automatic, 1 = never split)")
    ap.add_argument("--encoder", type=int, default=0,
                    help="0 = four-kernel encoder, 1 = single-pass encoder where it applies")
    ap.add_argument("--autotune", type=int, default=1,
                    help="pick chunk size, lanes, table width, CTAs/SM on a sample first")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--e2e-segment-mb", type=int, default=512,
                    help="container bytes per decode launch in the load plan")
    ap.add_argument("--per-tensor", type=int, default=1)
    ap.add_argument("--cpu-sample-mb", type=int, default=384)
    ap.add_argument("--layers", type=int, default=32, help="decoder layers (32 = 8B class)")
    ap.add_argument("--vocab", type=int, default=128256, help="embedding/head rows")
    ap.add_argument("--workload", default="checkpoint",
                    choices=["checkpoint", "serve", "plain", "fp32", "fp16", "delta",
                             "clean_fp32", "clean_fp16"])
    ap.add_argument("--delta-layers", type=int, default=24,
                    help="layers of the delta workload (24 = the 1.7B-parameter configuration)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-budget-gb", type=int, default=40)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-rate", type=float, default=200.0,
                    help="request arrivals per second (the served-stream workload: 200)")
    ap.add_argument("--ref-sample-mb", type=int, default=48)
    ap.add_argument("--split", type=int, default=0,
                    help="ranks decode disjoint chunk ranges of one checkpoint (strong scaling) "
                         "instead of each its own checkpoint")
    ap.add_argument("--configs", type=int, default=1,
                    help="also measure the checkpoint delta and a shortened served stream")
    ap.add_argument("--configs-serve-requests", type=int, default=400,
                    help="requests of the served stream measured with the default workload")
    ap.add_argument("--autotune-cache", type=int, default=0,
                    help="reuse a cached autotuner result instead of sweeping again")
    ap.add_argument("--autotune-log", default="",
                    help="write the autotuner's per-candidate table (JSON) here")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload in ("plain", "fp32", "fp16", "delta", "clean_fp32", "clean_fp16"):
        return run_tensors(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
