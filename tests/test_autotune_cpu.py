"""The autotuner's cache and the library's use of it (CPU only).

The tuner keeps its winner per (GPU, dtype, size class of the workload); the
Python API then takes that setting when a batched compressor is given no chunk
size or a decode plan no tuning.  Checked here without a GPU: the key, the
lookup by the workload's size class, and the concurrent-writer-safe save."""
from __future__ import annotations

import json
import os

from paper_2411_05239_gb300 import autotune as AT
from paper_2411_05239_gb300 import zipnn as Z


def test_cached_setting_is_found_by_workload_size(tmp_path, monkeypatch):
    monkeypatch.setenv("ZIPNN_TUNE_CACHE", str(tmp_path / "tune.json"))
    assert AT.cached(Z.BF16, 16_060_514_304) is None
    entry = {"chunk_bytes": 262144, "lanes": 512, "lut_bits": 12, "threads": 256,
             "ctas_per_sm": 3, "decode_gbs": 2700.0}
    AT.save_cache({AT.key(Z.BF16, 16_060_514_304): entry})
    assert not [f for f in os.listdir(tmp_path) if f.endswith(".tmp")]
    assert json.load(open(tmp_path / "tune.json"))
    # the same size class (2^33 bytes) finds it, another class or dtype does not
    assert Z.tuned_settings(Z.BF16, 10_000_000_000) == entry
    assert Z.tuned_settings(Z.BF16, 1 << 30) is None
    assert Z.tuned_settings(Z.FP32, 16_060_514_304) is None
    assert AT.size_class(16_060_514_304) == "2^33"
    assert AT.size_class(1) == "2^16"            # small workloads share one class


def test_unreadable_cache_reads_as_empty(tmp_path, monkeypatch):
    p = tmp_path / "tune.json"
    p.write_text("{not json")
    monkeypatch.setenv("ZIPNN_TUNE_CACHE", str(p))
    assert AT.load_cache() == {}
    assert Z.tuned_settings(Z.BF16, 1 << 34) is None
