"""Autotuner for batched launches.

Times the launch shapes a batched run can take on a sample of the actual
requests (CUDA events, median of a few repeats) and keeps the fastest:
  - sssp_threads: threads per search CTA (256 or 512);
  - chunk: instances per batched launch (a run over more instances than
    this is split into several launches; 2^30 means all at once).
Results are cached per (GPU name, size bucket) in memory and optionally in a
JSON file, so a serving process tunes each bucket once.
"""
from __future__ import annotations

import json
import os
import statistics

_cache: dict = {}


def _bucket(mats) -> str:
    import math
    nmax = max(int(S.shape[0]) for S in mats)
    return f"n<=2^{math.ceil(math.log2(max(nmax, 4)))}"


def tune_batch(ctx, mats, mode: str = "corr", prefix: int = 1, chunks=(32, 64, 1 << 30),
               threads=(256, 512), repeats: int = 3, cache_path: str | None = None) -> dict:
    """Pick {sssp_threads, chunk} for batched runs of matrices like ``mats``."""
    import torch
    import paper_2408_09399_gb300 as T
    key = f"{torch.cuda.get_device_name()}|{_bucket(mats)}|{mode}{prefix}"
    if key in _cache:
        return _cache[key]
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            disk = json.load(f)
        if key in disk:
            _cache[key] = disk[key]
            return disk[key]
    best = None
    cand = sorted(set(min(c, len(mats)) for c in chunks))
    for th in threads:
        for ch in cand:
            times = []
            for _ in range(repeats):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                for i in range(0, len(mats), ch):
                    T.tmfg_batch_run(ctx, mats[i:i + ch], mode, prefix, apsp=True,
                                     sssp_threads=th)
                b.record()
                T.tmfg_sync_status(ctx)
                times.append(a.elapsed_time(b))
            t = statistics.median(times)
            if best is None or t < best["ms"]:
                # a chunk that covered the whole sample means "all at once"
                best = {"sssp_threads": th, "chunk": ch if ch < len(mats) else 1 << 30, "ms": t}
    _cache[key] = best
    if cache_path:
        disk = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                disk = json.load(f)
        disk[key] = best
        with open(cache_path, "w") as f:
            json.dump(disk, f, indent=1)
    return best
