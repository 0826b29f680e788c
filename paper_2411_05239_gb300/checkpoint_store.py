"""Periodic-base checkpoint store over the XOR-delta codec (ZipNN Sec. 4.2,
"Periodic Base").

A training run saves checkpoints 0, 1, 2, ...; every `period`-th one is stored
whole (a base, compressed standalone) and the others as XOR deltas, so that a
checkpoint is recovered from a bounded amount of data.  Two policies, as the
paper describes them:

* ``"chain"``: checkpoint i is a delta against checkpoint i - 1; recovering it
  decodes the last base and then every delta up to i (chains of at most
  period - 1 deltas).
* ``"base"``: checkpoint i is a delta against the last base; recovering it
  decodes the base and one delta (never a chain), at the price of deltas taken
  across up to period - 1 checkpoints.

The store is host-side bookkeeping: which entry is a base, which entry each
delta refers to, and the order in which to decode.  The codec is injected
(``codec``), so the policy is testable without a GPU; `GpuCodec` is the one the
package uses, built on the batched compressor and decoder.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Protocol


class Codec(Protocol):
    def compress(self, tensors: list, bases: list | None) -> list: ...
    def decompress(self, containers: list, bases: list | None) -> list: ...
    def nbytes(self, containers: list) -> int: ...


@dataclass
class Entry:
    index: int
    ref: int | None          # checkpoint this one is a delta against (None: base)
    containers: list = field(default_factory=list)

    @property
    def is_base(self) -> bool:
        return self.ref is None


class CheckpointStore:
    """Stores checkpoints (each a list of tensors) with a base every `period`
    checkpoints; `policy` is "chain" or "base" (see the module docstring)."""

    def __init__(self, codec: Codec, period: int = 10, policy: str = "chain"):
        if period < 1:
            raise ValueError("period must be >= 1")
        if policy not in ("chain", "base"):
            raise ValueError("policy must be 'chain' or 'base'")
        self.codec = codec
        self.period = period
        self.policy = policy
        self.entries: list[Entry] = []
        # the reference of the next delta, as a private copy (training updates
        # the caller's tensors in place): the newest checkpoint ("chain") or
        # the newest base ("base")
        self._ref: list | None = None

    # -- policy ------------------------------------------------------------
    def ref_of(self, i: int) -> int | None:
        """Checkpoint that checkpoint i is stored against (None: stored whole)."""
        if i % self.period == 0:
            return None
        return i - 1 if self.policy == "chain" else i - i % self.period

    def decode_path(self, i: int) -> list[int]:
        """Entries to decode, base first, to recover checkpoint i."""
        path = [i]
        while self.ref_of(path[-1]) is not None:
            path.append(self.ref_of(path[-1]))
        return path[::-1]

    # -- store / load ------------------------------------------------------
    def put(self, tensors: list) -> Entry:
        i = len(self.entries)
        ref = self.ref_of(i)
        cont = self.codec.compress(tensors, None if ref is None else self._ref)
        e = Entry(i, ref, cont)
        self.entries.append(e)
        if ref is None or self.policy == "chain":
            self._ref = [_snapshot(t) for t in tensors]
        return e

    def get(self, i: int) -> list:
        if not 0 <= i < len(self.entries):
            raise IndexError(i)
        cur = None
        for k in self.decode_path(i):
            e = self.entries[k]
            cur = self.codec.decompress(e.containers, None if e.is_base else cur)
        return cur

    def stored_bytes(self) -> int:
        return sum(self.codec.nbytes(e.containers) for e in self.entries)


def _snapshot(t):
    return t.clone() if hasattr(t, "clone") else t.copy()


class GpuCodec:
    """The package's codec: batched compression of a checkpoint's tensors (XOR
    deltas when bases are given) and one persistent batched decode."""

    def __init__(self, chunk_bytes: int | None = None):
        from . import zipnn as Z
        self.Z = Z
        self.chunk_bytes = chunk_bytes or Z.DEFAULT_CHUNK

    def compress(self, tensors: list, bases: list | None) -> list:
        return [self.Z.compress(t, chunk_bytes=self.chunk_bytes,
                                base=None if bases is None else b)
                for t, b in zip(tensors, bases if bases is not None else [None] * len(tensors))]

    def decompress(self, containers: list, bases: list | None) -> list:
        import torch
        outs = [torch.empty(c.orig_nbytes, dtype=torch.uint8, device="cuda") for c in containers]
        self.Z.batch_decompress(containers, outs, bases=bases)
        self.Z.sync_status()
        dts = [self.Z.CODE_TO_TORCH[c.zs.dtype] for c in containers]
        return [o.view(dt) for o, dt in zip(outs, dts)]

    def nbytes(self, containers: list) -> int:
        return sum(c.nbytes for c in containers)

