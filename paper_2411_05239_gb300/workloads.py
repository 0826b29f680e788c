"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures real Hugging Face models (ZipNN Sec. 3.3 Table 2, Sec. 5.2
Table 3: "1GB from the middle of the model"); none are available here, so these
generators stand in for them with the same dtypes, shapes and value
distributions.  This module holds no codec arithmetic: it only draws numbers.
Both the CUDA path and the CPU oracle consume the exact bytes produced here.

Every generator takes a ``device``; drawing on the GPU is fast for the large
configurations, drawing on the CPU gives the same recipe with different numbers
(torch's CPU and CUDA generators differ), which is fine because each test hands
the same bytes to both sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def gaussian(n: int, std: float, seed: int, dtype=torch.bfloat16, device="cpu") -> torch.Tensor:
    """i.i.d. N(0, std) drawn in fp32, rounded to ``dtype`` (round to nearest even)."""
    g = _gen(seed, device)
    return (torch.randn(n, generator=g, device=device, dtype=torch.float32) * std).to(dtype)


# ---------------------------------------------------------------------------
# Plain single tensor: 4,194,304 BF16 values, N(0, 0.02), seed 0.
def plain_bf16(n: int = 4_194_304, seed: int = 0, device="cpu") -> torch.Tensor:
    return gaussian(n, 0.02, seed, torch.bfloat16, device)


# ---------------------------------------------------------------------------
# FP32 8192x8192: each row N(0, s_r), s_r log-uniform in [1e-3, 1e-1]; 2% exact
# zeros; seed 1.  The row scales are drawn first, then the values, then the mask.
def rowscaled_fp32(rows: int = 8192, cols: int = 8192, seed: int = 1, device="cpu") -> torch.Tensor:
    g = _gen(seed, device)
    u = torch.rand(rows, generator=g, device=device, dtype=torch.float32)
    s = torch.pow(10.0, -3.0 + 2.0 * u)
    x = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float32) * s[:, None]
    mask = torch.rand(rows, cols, generator=g, device=device, dtype=torch.float32) < 0.02
    x[mask] = 0.0
    return x.reshape(-1)


# ---------------------------------------------------------------------------
# "Clean" models (Sec. 3.2): parameters held in a wider type than the precision
# they carry.  FP32 holding BF16 values has its 16 low bits zero (the T5 rows of
# the byte-grouping size table); FP16 holding BF16 values has the 3 low fraction
# bits of every normal number zero.  N(0, 0.02) drawn as BF16; seeds 5 and 6;
# 67,108,864 values (256 MiB FP32, 128 MiB FP16).
def clean_fp32_from_bf16(n: int = 67_108_864, seed: int = 5, device="cpu") -> torch.Tensor:
    return gaussian(n, 0.02, seed, torch.bfloat16, device).to(torch.float32)


def clean_fp16_from_bf16(n: int = 67_108_864, seed: int = 6, device="cpu") -> torch.Tensor:
    return gaussian(n, 0.02, seed, torch.bfloat16, device).to(torch.float16)


# ---------------------------------------------------------------------------
# 8B-class decoder-only checkpoint in BF16 (Llama-3.1-8B shapes): 32 layers of
# q,o 4096x4096, k,v 1024x4096, gate,up 14336x4096, down 4096x14336, two RMSNorm
# vectors of ones; embedding and head 128256x4096.  Weights N(0, 0.02/sqrt(2l+1))
# for layer l, N(0, 0.02) for embedding and head; seed 2.
@dataclass
class TensorSpec:
    name: str
    shape: tuple
    std: float          # 0.0 marks an all-ones norm vector

    @property
    def numel(self) -> int:
        return int(np.prod(self.shape))


def llama8b_specs(n_layers: int = 32, hidden: int = 4096, kv: int = 1024, ffn: int = 14336,
                  vocab: int = 128256) -> list[TensorSpec]:
    specs = [TensorSpec("embed", (vocab, hidden), 0.02)]
    for layer in range(n_layers):
        s = 0.02 / math.sqrt(2 * layer + 1)
        specs += [
            TensorSpec(f"l{layer}.q", (hidden, hidden), s),
            TensorSpec(f"l{layer}.k", (kv, hidden), s),
            TensorSpec(f"l{layer}.v", (kv, hidden), s),
            TensorSpec(f"l{layer}.o", (hidden, hidden), s),
            TensorSpec(f"l{layer}.gate", (ffn, hidden), s),
            TensorSpec(f"l{layer}.up", (ffn, hidden), s),
            TensorSpec(f"l{layer}.down", (hidden, ffn), s),
            TensorSpec(f"l{layer}.norm1", (hidden,), 0.0),
            TensorSpec(f"l{layer}.norm2", (hidden,), 0.0),
        ]
    specs.append(TensorSpec("head", (vocab, hidden), 0.02))
    return specs


def checkpoint_bf16(specs: list[TensorSpec], seed: int = 2, device="cpu") -> list[torch.Tensor]:
    g = _gen(seed, device)
    out = []
    for sp in specs:
        if sp.std == 0.0:
            out.append(torch.ones(sp.numel, dtype=torch.bfloat16, device=device))
        else:
            t = torch.randn(sp.numel, generator=g, device=device, dtype=torch.float32)
            out.append(t.mul_(sp.std).to(torch.bfloat16))
            del t
    return out


# ---------------------------------------------------------------------------
# Checkpoint delta: base = 24 layers of 2048x2048 (x4) and 2048x8192 (x3) plus a
# 50,000x2048 embedding, N(0, 0.02); next = bf16(base + N(0, 1e-4)) on a random
# 30% of entries, else identical; seed 3.
def delta_specs(n_layers: int = 24, hidden: int = 2048, ffn: int = 8192,
                vocab: int = 50_000) -> list[TensorSpec]:
    specs = [TensorSpec("embed", (vocab, hidden), 0.02)]
    for layer in range(n_layers):
        for nm in ("q", "k", "v", "o"):
            specs.append(TensorSpec(f"l{layer}.{nm}", (hidden, hidden), 0.02))
        for nm in ("gate", "up", "down"):
            specs.append(TensorSpec(f"l{layer}.{nm}", (hidden, ffn), 0.02))
    return specs


def delta_pair(numel: int, seed: int = 3, device="cpu", frac: float = 0.3,
               noise: float = 1e-4) -> tuple[torch.Tensor, torch.Tensor]:
    """(next, base) of ``numel`` BF16 values as one flat pair."""
    g = _gen(seed, device)
    base = (torch.randn(numel, generator=g, device=device, dtype=torch.float32) * 0.02)
    base = base.to(torch.bfloat16)
    pert = torch.randn(numel, generator=g, device=device, dtype=torch.float32) * noise
    mask = torch.rand(numel, generator=g, device=device, dtype=torch.float32) < frac
    nxt = torch.where(mask, (base.float() + pert).to(torch.bfloat16), base)
    return nxt, base


# ---------------------------------------------------------------------------
# Served stream: Poisson arrivals at 200 req/s; 70% compress / 30% decompress;
# dtype BF16/FP16/FP32 (60/20/20); size log-uniform in [64 KiB, 2 GiB] rounded
# down to the element size; 15% deltas against a resident base; seed 4.
@dataclass
class Request:
    rid: int
    t_arrival: float
    op: str            # "compress" or "decompress"
    dtype: str         # "bf16", "fp16", "fp32"
    nbytes: int
    delta: bool


def request_trace(n: int = 2000, seed: int = 4, rate: float = 200.0,
                  lo: int = 64 << 10, hi: int = 2 << 30) -> list[Request]:
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps) - gaps[0]
    ops = np.where(rng.random(n) < 0.7, "compress", "decompress")
    dt = rng.choice(["bf16", "fp16", "fp32"], size=n, p=[0.6, 0.2, 0.2])
    sizes = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))).astype(np.int64)
    deltas = rng.random(n) < 0.15
    es = {"bf16": 2, "fp16": 2, "fp32": 4}
    return [Request(i, float(t[i]), str(ops[i]), str(dt[i]),
                    int(sizes[i] // es[str(dt[i])] * es[str(dt[i])]), bool(deltas[i]))
            for i in range(n)]


TORCH_DTYPE = {"bf16": torch.bfloat16, "fp16": torch.float16, "fp32": torch.float32}


def serve_inputs(trace: list[Request], device="cuda"):
    """Input tensors of a request trace: one pool per dtype, sized for the
    largest request, holding plain N(0, 0.02) values and a delta pair made as
    in ``delta_pair`` (a 30% perturbation at 1e-4, cast to the dtype); request
    r takes the first r.nbytes bytes of its dtype's pool.  Returns a function
    mapping a request to (tensor, base or None)."""
    maxb = max(r.nbytes for r in trace) if trace else 0
    pools = {}
    for k, (dt, tdt) in enumerate(TORCH_DTYPE.items()):
        es = torch.tensor([], dtype=tdt).element_size()
        n = maxb // es + 1
        nxt, base = delta_pair(n, seed=40 + k, device=device)
        plain = gaussian(n, 0.02, seed=50 + k, dtype=tdt, device=device)
        if tdt != torch.bfloat16:
            nxt, base = nxt.to(tdt), base.to(tdt)
        pools[dt] = (plain, nxt, base)

    def inputs(r: Request):
        es = {"bf16": 2, "fp16": 2, "fp32": 4}[r.dtype]
        n = r.nbytes // es
        plain, nxt, base = pools[r.dtype]
        return (nxt[:n], base[:n]) if r.delta else (plain[:n], None)

    return inputs
