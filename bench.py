"""Benchmark: TMFG + APSP on the n=20000 time-series workload (one GB300).

A step is one pass of the whole hot path over one input matrix S (n=20000,
float32, Pearson correlations of 20000 planted-factor series of length 2000,
50 clusters, Student-t(4) noise): validation, exact row sums and the per-row
sort, the heap-tmfg insertion loop, CSR + exact APSP, and the hub-based
approximate APSP.  S (1.6 GB) is larger than L2, so successive steps do not
run from cache.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n N]

Rank 0 prints one JSON line.  With torchrun (N>1) every rank solves its own
instance (no data-path collective; the greedy loop does not shard) and the
time is the max over ranks.  ``--impl reference`` times the CPU oracle (the
only reference implementation of this method that exists here) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TMFG+APSP ms at n=20k"
KERNELS_PER_STEP = 14  # rowsort, loop; 4 exact-APSP kernels; 8 approximate-APSP kernels


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_input(n, device):
    from paper_2408_09399_gb300 import workloads as W
    S, _ = W.config_similarity(3, device=device, n=n)
    return S


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def run_ours(args, rank, world, local):
    import torch
    import paper_2408_09399_gb300 as T
    from paper_2408_09399_gb300 import build as B

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n = args.n
    S = make_input(n, f"cuda:{local}")
    ctx = T.tmfg_create(local)
    stream = torch.cuda.current_stream()
    out = {"order": torch.empty(n, dtype=torch.int32, device=dev),
           "edges": torch.empty((3 * n - 6, 2), dtype=torch.int32, device=dev),
           "ins_face": torch.empty((n - 4, 3), dtype=torch.int32, device=dev),
           "bubble_parent": torch.empty(n - 3, dtype=torch.int32, device=dev)}
    D = torch.empty((n, n), dtype=torch.float32, device=dev)
    Da = torch.empty((n, n), dtype=torch.float32, device=dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(times=None):
        e0, e1, e2, e3 = ev(), ev(), ev(), ev()
        e0.record(stream)
        T.tmfg_build(ctx, S, "heap", 1, out=out, stream=stream)
        e1.record(stream)
        T.tmfg_apsp(ctx, S, out["edges"], D=D, stream=stream)
        e2.record(stream)
        T.tmfg_apsp(ctx, S, out["edges"], approx=True, D=Da, stream=stream)
        e3.record(stream)
        if times is not None:
            times.append((e0, e1, e2, e3))

    for _ in range(args.warmup):
        step()
    T.tmfg_sync_status(ctx, stream)
    loop_ns = T.tmfg_last_stats(ctx)["loop_ns"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times = []
    with ClockSampler(local) as clk:
        t0 = ev()
        t1 = ev()
        t0.record(stream)
        for _ in range(args.steps):
            step(times)
        t1.record(stream)
        torch.cuda.synchronize()
    T.tmfg_sync_status(ctx, stream)
    stats = T.tmfg_last_stats(ctx)
    total_ms = t0.elapsed_time(t1)
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
        dist.barrier()
    ms_step = total_ms / args.steps
    ph = np.array([[a.elapsed_time(b), b.elapsed_time(c), c.elapsed_time(d)]
                   for a, b, c, d in times])
    tmfg_ms, apsp_ms, apsx_ms = ph.mean(axis=0).tolist()
    loop_ms = stats["loop_ns"] / 1e6

    # row sort alone (same kernel as inside tmfg_build), for the phase split
    idx = torch.empty((n, ((n - 1) + 7) // 8 * 8), dtype=torch.int16, device=dev)
    rs = torch.empty(n, dtype=torch.int64, device=dev)
    T.tmfg_row_sort(ctx, S, idx, rs, stream=stream)
    sort_times = []
    for _ in range(3):
        a, b = ev(), ev()
        a.record(stream)
        T.tmfg_row_sort(ctx, S, idx, rs, stream=stream)
        b.record(stream)
        sort_times.append((a, b))
    T.tmfg_sync_status(ctx, stream)
    sort_ms = float(np.mean([a.elapsed_time(b) for a, b in sort_times]))

    # roofline of the dominant HBM-bound kernel and of the whole step
    hbm_peak, peak_kind = measured_peaks()
    phases = {"sort_rowsum_ms": sort_ms, "loop_ms": loop_ms, "tmfg_total_ms": tmfg_ms,
              "apsp_exact_ms": apsp_ms, "apsp_approx_ms": apsx_ms}
    # algorithmic bytes: sort reads S (4n^2) and writes the index rows (2n^2);
    # each APSP writes D (4n^2)
    alg = {"sort": 6.0 * n * n, "apsp_exact": 4.0 * n * n, "apsp_approx": 4.0 * n * n}
    cand = {"sort": sort_ms, "apsp_exact": apsp_ms, "apsp_approx": apsx_ms}
    dom = max(cand, key=cand.get)
    achieved = alg[dom] / (cand[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm_peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "traffic": None,
                "note": "the heap insertion loop (loop_ms) is a chain of n-4 dependent steps "
                        "bound by memory latency, not bandwidth; it is reported as ns/step"}

    e2e = None
    if not args.no_e2e and rank == 0:
        Sh = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        Sh.copy_(S)
        Dh = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        Dah = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
        Eh = torch.empty((3 * n - 6, 2), dtype=torch.int32, pin_memory=True)
        Sd = torch.empty_like(S)

        def e2e_step():
            Sd.copy_(Sh, non_blocking=True)
            T.tmfg_build(ctx, Sd, "heap", 1, out=out, stream=stream)
            T.tmfg_apsp(ctx, Sd, out["edges"], D=D, stream=stream)
            T.tmfg_apsp(ctx, Sd, out["edges"], approx=True, D=Da, stream=stream)
            Eh.copy_(out["edges"], non_blocking=True)
            Dh.copy_(D, non_blocking=True)
            Dah.copy_(Da, non_blocking=True)

        e2e_step()
        T.tmfg_sync_status(ctx, stream)
        a, b = ev(), ev()
        k = max(1, min(args.steps, 3))
        a.record(stream)
        for _ in range(k):
            e2e_step()
        b.record(stream)
        T.tmfg_sync_status(ctx, stream)
        e2e = {"value": round(a.elapsed_time(b) / k, 3), "unit": "ms",
               "h2d_bytes_per_step": 4 * n * n,
               "d2h_bytes_per_step": 2 * 4 * n * n + 4 * 2 * (3 * n - 6)}

    result = {
        "metric": METRIC, "value": round(ms_step, 3), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"n={n} T=2000 50 planted clusters, Student-t(4) noise, "
                               "float32 Pearson S; heap-tmfg + exact APSP + approximate APSP",
                   "n": n, "tmfg": "heap (P=1)", "apsp": "exact + approximate (ceil(sqrt n) hubs, "
                   "radius factor 2)", "l2": "inputs larger than L2 (S is 1.6 GB)",
                   "parallelism": f"replicas x{world}"},
        "phases": {k: round(v, 3) for k, v in phases.items()},
        "loop_ns_per_insertion": round(stats["loop_ns"] / max(1, n - 4), 1),
        "loop_stats": stats,
        "roofline": roofline,
        "algorithmic_bytes_per_step": int(14 * n * n),
        "step_hbm_frac": round(14.0 * n * n / (ms_step * 1e-3) / 1e9 / hbm_peak, 4),
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": KERNELS_PER_STEP * args.steps,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(S.cpu().numpy(), out, n)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return result


def cpu_baseline(Sn, out, n, budget_s: float = 25.0):
    """The oracle on a bounded sample of the same workload, scaled to the
    full step: sorted rows for a sample of rows, the full heap insertion loop
    is not sampled (it needs every row); exact SSSP from sampled sources;
    approximate APSP as the hub searches plus bounded searches from sampled
    sources.  Every sampled part is scaled by n / sample size."""
    import oracle
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    rows = np.arange(0, n, max(1, n // 64))[:64].astype(np.int32)
    oracle.rowsort_rows(Sn, rows)
    t_sort = (time.perf_counter() - t) * n / len(rows)
    edges = out["edges"].cpu().numpy()  # graph shape only: the oracle's own edges below
    del edges
    # the oracle's own TMFG on a sub-problem would change the workload, so
    # the loop is timed with the oracle's corr/heap code on the full matrix
    # only when that fits the budget; otherwise it is left out and said so
    t = time.perf_counter()
    ref_edges = None
    loop_note = "heap loop timed in full"
    if n <= 6000:
        ref = oracle.tmfg(Sn, "heap")
        ref_edges = ref["edges"]
        t_tmfg = time.perf_counter() - t
    else:
        # sort the full matrix would dominate the budget; time the loop on a
        # leading principal submatrix of 4000 series and scale by (n/4000)^1
        sub = np.ascontiguousarray(Sn[:4000, :4000])
        ref = oracle.tmfg(sub, "heap")
        ref_edges = ref["edges"]
        t_tmfg = (time.perf_counter() - t) * (n / 4000.0) ** 2
        loop_note = "heap TMFG timed on the 4000x4000 leading submatrix, scaled by (n/4000)^2"
    src = np.arange(0, 4000, 4000 // 64)[:64].astype(np.int32)
    t = time.perf_counter()
    oracle.sssp_rows(np.ascontiguousarray(Sn[:4000, :4000]), ref_edges, src, prec=32)
    t_apsp = (time.perf_counter() - t) * (4000 / len(src)) * (n / 4000.0) ** 2
    t_total = t_sort + t_tmfg + 2 * t_apsp
    return {"value": round(t_total * 1e3, 1), "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": f"64 sorted rows of the n={n} matrix (scaled x{n // 64}); {loop_note}; "
                      "64 exact SSSP rows on the submatrix TMFG scaled to n^2 work (counted "
                      "twice for the exact and approximate APSP)",
            "parts_ms": {"sort": round(t_sort * 1e3, 1), "tmfg": round(t_tmfg * 1e3, 1),
                         "apsp": round(t_apsp * 1e3, 1)}}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    n = args.n
    Sn = make_input(n, "cpu")
    times = []
    for _ in range(args.warmup + args.steps):
        t = time.perf_counter()
        base = cpu_baseline(Sn, {"edges": _Dummy()}, n)
        times.append(time.perf_counter() - t)
        last = base
    v = last["value"]
    return {"metric": METRIC, "value": v, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64/f32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"n={n} T=2000 50 planted clusters, Student-t(4) noise, "
                                   "float32 Pearson S; heap-tmfg + exact APSP + approximate APSP",
                       "n": n},
            "cpu_baseline": {k: last[k] for k in ("kind", "cores", "sample")} | {"value": v,
                                                                                 "unit": "ms"},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


class _Dummy:
    def cpu(self):
        return self

    def numpy(self):
        return np.zeros((0, 2), np.int32)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        r = run_reference(args, rank, world)
    else:
        r = run_ours(args, rank, world, local)
    if rank == 0 and r is not None:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
