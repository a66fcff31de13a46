"""Autotuner for batched PW evaluations: picks the kernel variant (tile shape
and TMA pipeline depth, see pw_variant_count in include/pw.h) by timing each
on the batch itself, and caches the winner per shape class in a JSON file.

Shape class of a batch: library version (variant numbering belongs to it),
arithmetic mode, number of domains, and the domains' sizes rounded to powers
of two (x, y, z) as a sorted histogram, so batches with similar geometry
reuse one measurement.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import pw

_lock = threading.Lock()


def default_cache_path() -> str:
    return os.environ.get("PW_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pw_gb300", "tune.json"))


def _p2(n: int) -> int:
    return 1 << max(0, math.ceil(math.log2(max(n, 1))))


def shape_class(mode: str, domains) -> str:
    hist = {}
    for d in domains:
        key = (_p2(d["nx"]), _p2(d["ny"]), _p2(d["u"].shape[0]))
        hist[key] = hist.get(key, 0) + 1
    parts = ",".join(f"{x}x{y}x{z}:{c}" for (x, y, z), c in sorted(hist.items()))
    return f"{pw.version()}|{mode}|n={len(domains)}|{parts}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def time_batch(batch, reps=5, warmup=2) -> float:
    """Mean ms per launch of a Batch (CUDA events on the current stream)."""
    import torch
    for _ in range(warmup):
        batch.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        batch.run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(domains, mode="paired", cache_path=None, reps=5, force=False):
    """Return (variant, record) for this batch, measuring every variant once
    per shape class and caching the result."""
    path = cache_path or default_cache_path()
    key = shape_class(mode, domains)
    with _lock:
        cache = _load(path)
        if not force and key in cache:
            return int(cache[key]["variant"]), cache[key]
    times = {}
    for v in range(pw.variant_count(mode)):
        b = pw.Batch(domains, mode, v)
        times[v] = time_batch(b, reps)
    best = min(times, key=times.get)
    rec = {"variant": best, "ms": {str(k): t for k, t in times.items()}}
    with _lock:
        cache = _load(path)
        cache[key] = rec
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return best, rec
