"""Autotuner for the launch shapes of the loop, the searches and batching.

Times the shapes a run can take on a sample of the actual work (CUDA
events, median of a few repeats) and keeps the fastest; every shape gives
the same results, so only the time decides:
  - loop: the corr-tmfg prefix-1 insertion loop's kernel (the general one,
    the prefix-1 one, or for single builds the cluster one), its threads per
    CTA, lanes per sorted-row refresh, copied index groups and cluster size
    (tmfg_loop_shape);
  - sssp_threads: threads per search CTA (256 or 512);
  - chunk: instances per batched launch (a run over more instances than
    this is split into several launches; 2^30 means all at once).
The search is coordinate-wise: the loop shape first (the other knobs at
their defaults), then the search threads, then the chunk.  Results are
cached per (GPU name, size bucket, work) in memory and optionally in a JSON
file, so a serving process tunes each bucket once.
"""
from __future__ import annotations

import json
import math
import os
import statistics

_cache: dict = {}

# candidate loop shapes (tmfg_set_loop_shape / tmfg_batch_config.loop)
LOOP_SHAPES = (
    {"kernel": 2},
    {"kernel": 1, "threads": 256, "probe_lanes": 8},
    {"kernel": 1, "threads": 256, "probe_lanes": 16},
    {"kernel": 1, "threads": 512, "probe_lanes": 16},
    {"kernel": 1, "threads": 256, "probe_lanes": 8, "stage_groups": -1},
)
# single builds may also run on a thread-block cluster (not in batches)
SINGLE_LOOP_SHAPES = LOOP_SHAPES + (
    {"kernel": 3, "cluster": 8, "probe_lanes": 32},
    {"kernel": 3, "cluster": 16, "probe_lanes": 16},
    {"kernel": 3, "cluster": 16, "probe_lanes": 32},
)


def _bucket(sizes) -> str:
    return f"n<=2^{math.ceil(math.log2(max(max(sizes), 4)))}"


def _time(fn, repeats: int) -> float:
    import torch
    times = []
    for _ in range(repeats):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def _cached(key, cache_path):
    if key in _cache:
        return _cache[key]
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            disk = json.load(f)
        if key in disk:
            _cache[key] = disk[key]
            return disk[key]
    return None


def _store(key, best, cache_path):
    _cache[key] = best
    if cache_path:
        disk = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                disk = json.load(f)
        disk[key] = best
        with open(cache_path, "w") as f:
            json.dump(disk, f, indent=1)


def _coordinate_search(run, count, chunks, threads, repeats):
    """run(loop_shape, sssp_threads, chunk) performs the work once."""
    tried = []

    def t_of(shape, th, ch):
        t = _time(lambda: run(shape, th, ch), repeats)
        tried.append({"loop": shape, "sssp_threads": th, "chunk": ch, "ms": round(t, 3)})
        return t

    all_at_once = 1 << 30
    shape = min(LOOP_SHAPES, key=lambda sh: t_of(sh, 512, all_at_once))
    th = min(threads, key=lambda x: t_of(shape, x, all_at_once))
    cand = sorted(set(min(c, count) for c in chunks))
    ch = min(cand, key=lambda c: t_of(shape, th, c))
    best_ms = min(r["ms"] for r in tried if r["loop"] == shape and r["sssp_threads"] == th and
                  r["chunk"] == ch)
    return {"loop": shape, "sssp_threads": th, "chunk": ch if ch < count else all_at_once,
            "ms": best_ms, "tried": len(tried)}


def tune_batch(ctx, mats, mode: str = "corr", prefix: int = 1, chunks=(32, 64, 1 << 30),
               threads=(256, 512), repeats: int = 3, cache_path: str | None = None) -> dict:
    """Pick {loop, sssp_threads, chunk} for batched TMFG + APSP runs of
    matrices like ``mats``."""
    import torch
    import paper_2408_09399_gb300 as T
    key = (f"{torch.cuda.get_device_name()}|batch|{_bucket([S.shape[0] for S in mats])}|"
           f"{mode}{prefix}")
    hit = _cached(key, cache_path)
    if hit:
        return hit

    def run(shape, th, ch):
        for i in range(0, len(mats), ch):
            T.tmfg_batch_run(ctx, mats[i:i + ch], mode, prefix, apsp=True, sssp_threads=th,
                             loop_shape=shape if mode == "corr" and prefix == 1 else None)
        T.tmfg_sync_status(ctx)

    best = _coordinate_search(run, len(mats), chunks, threads, repeats)
    _store(key, best, cache_path)
    return best


def tune_pipeline(ctx, series, ks, precision: str = "bf16x3", chunks=(64, 256, 1 << 30),
                  threads=(256, 512), repeats: int = 2, cache_path: str | None = None) -> dict:
    """Pick {loop, sssp_threads, chunk} for tmfg_pipeline_run over requests
    like (series, ks)."""
    import torch
    import paper_2408_09399_gb300 as T
    key = (f"{torch.cuda.get_device_name()}|pipeline|{_bucket([X.shape[0] for X in series])}|"
           f"{precision}")
    hit = _cached(key, cache_path)
    if hit:
        return hit
    outs = [T._pipeline_outputs(X.shape[0], X.device) for X in series]

    def run(shape, th, ch):
        for i in range(0, len(series), ch):
            T.tmfg_pipeline_run(ctx, series[i:i + ch], ks[i:i + ch], precision,
                                outs=outs[i:i + ch], sssp_threads=th, loop_shape=shape)
        T.tmfg_sync_status(ctx)

    best = _coordinate_search(run, len(series), chunks, threads, repeats)
    _store(key, best, cache_path)
    return best


def tune_loop(ctx, S, mode: str = "corr", prefix: int = 1, repeats: int = 2,
              apply: bool = True, cache_path: str | None = None) -> dict:
    """Pick the loop shape for single builds of matrices like S (corr-tmfg
    prefix 1; other modes have one shape) and, with ``apply``, set it on the
    context.  Returns {loop, ms, tried: [{loop, ms}]}."""
    import torch
    import paper_2408_09399_gb300 as T
    if mode != "corr" or prefix != 1:
        return {"loop": None, "ms": None, "tried": []}
    n = int(S.shape[0])
    key = f"{torch.cuda.get_device_name()}|loop|{_bucket([n])}|{S.dtype}"
    best = _cached(key, cache_path)
    if not best:
        tried = []
        for sh in SINGLE_LOOP_SHAPES:
            T.tmfg_set_loop_shape(ctx, sh)

            def run():
                T.tmfg_build(ctx, S, mode, prefix)
                T.tmfg_sync_status(ctx)

            try:
                tried.append({"loop": sh, "ms": round(_time(run, repeats), 3)})
            except T.TmfgError:
                continue  # a shape that does not hold this n
        win = min(tried, key=lambda r: r["ms"])
        best = {"loop": win["loop"], "ms": win["ms"], "tried": tried}
        _store(key, best, cache_path)
    T.tmfg_set_loop_shape(ctx, best["loop"] if apply else None)
    return best
