"""Benchmark of the key-only Top-K offload (and, as they land, the join probe,
the batched executor and the gated serving loop) on GB300.

One step = one Top-K query, ORDER BY key DESC LIMIT K, over N = 2^28 int64
keys drawn uniformly over the full int64 range (K = 1000 by default), the
Top-K-at-scale workload.  ``value`` is keys/s with the keys resident in HBM
(one cooperative kernel launch per step); ``e2e`` is the same query through
the public blocking call with the keys in pinned host memory, so the key-only
H2D copy and the D2H of the K (key, row-id) results are inside the timed
region.  The keys (2 GiB) are larger than L2 (129 MB), so no flush is needed
between steps.

``--impl reference`` times the CPU oracle (a full stable sort then the first
K, single thread) on a bounded sample of the same workload instead.
Under torchrun each rank runs an independent replica on its own GPU ("replicas
only": the selection needs no exchange); rank 0 prints the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Top-K Gkeys/s & join probes/s (% HBM peak); batched vs per-query; gated P99"


# DRAM bytes (read + write) per input key of the Top-K filter kernel, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of that kernel at
# 2^26 uniform keys with explicit row-ids, K = 1000, register filter; the
# traffic of a full launch is this figure times n (the reads are the keys and
# the candidates' row-ids, the writes the candidates, all in proportion to n).
# Valid only for that configuration.
FILTER_DRAM_BYTES_PER_KEY = {"i64": 546_427_136 / 2**26, "f32": 277_938_944 / 2**26}


def _kernel_pass(ctx, steps, launch):
    """Run `launch` `steps` more times with per-kernel CUDA events on the
    library's stream; the mean device time of each kernel (ms)."""
    ctx.time_kernels(True)
    acc = {}
    for _ in range(steps):
        launch()
        for nm, v in ctx.kernel_ms().items():
            if v >= 0:
                acc.setdefault(nm, []).append(v)
    ctx.time_kernels(False)
    return {nm: float(np.mean(v)) for nm, v in acc.items()}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks.mem,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mem, mx, reasons = [], [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
                mem.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "mem_mhz": float(np.median(mem)),
                "mem_mhz_min": float(np.min(mem)), "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    from paper_2601_19911_gb300 import replicas
    return replicas.env()


def _max_over_ranks(x: float, world: int) -> float:
    from paper_2601_19911_gb300 import replicas
    return replicas.max_over_ranks(x, world, device="cuda")


def _barrier(world):
    from paper_2601_19911_gb300 import replicas
    replicas.barrier(world)


def cpu_baseline(n_full: int, k: int, seconds: float = 12.0):
    """The oracle as it stands, single thread, on a bounded sample of the
    workload (the first 2^22 keys of the same column), scaled to keys/s."""
    import oracle
    from paper_2601_19911_gb300 import datagen
    ns = 1 << 22
    keys = datagen.topk_keys(ns, "uniform", "i64", seed=1)
    oracle.topk(keys[:1000], k, oracle.DESC)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.topk(keys, k, oracle.DESC)
        reps += 1
        el = time.perf_counter() - t0
        if el > seconds:
            break
    per = el / reps
    return {"value": ns / per / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
            "sample": f"{reps} x oracle Top-K (stable sort, first K={k}) of {ns} uniform int64 keys, "
                      f"1 thread; {per * 1e3:.1f} ms each"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    k = args.k
    import oracle
    from paper_2601_19911_gb300 import datagen
    ns = 1 << 22
    keys = datagen.topk_keys(ns, "uniform", "i64", seed=1)
    for _ in range(args.warmup):
        oracle.topk(keys, k, oracle.DESC)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.topk(keys, k, oracle.DESC)
    el = time.perf_counter() - t0
    per = el / args.steps
    v = ns / per / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gkeys/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"topk_i64_uniform_n{ns}_k{k}_desc (bounded sample of the 2^28 workload)",
                       "n": ns, "k": k},
            "cpu_baseline": {"value": v, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed steps of the oracle on {ns} keys",
                             "host": _host_info()},
            "e2e": {"value": v, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def join_leg(args, ctx, torch, world):
    """Probe of 2^log2p int64 keys against a resident table of 2^log2b build
    rows; one probe launch per step.  Returns the join sub-object."""
    from paper_2601_19911_gb300 import datagen, olap
    mult, dist, hit = args.join_cell.split(",")
    hit = float(hit)
    nb, npr = 1 << args.join_log2b, 1 << args.join_log2p
    b = datagen.join_build(nb, mult, seed=2)
    p = datagen.join_probe(npr, b, hit, dist, seed=2)
    need = p.expected_pairs(b)
    dbk = torch.from_numpy(b.keys).cuda()
    stream = torch.cuda.ExternalStream(ctx.stream)
    # build (timed once, after one warm build)
    ctx.join_build(dbk).free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    table = ctx.join_build(dbk)
    build_s = time.perf_counter() - t0
    dk = torch.from_numpy(p.keys).cuda()
    out = torch.empty((need, 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(max(3, args.warmup)):
        ctx.join_probe_async(table, dk, out, need, cnt)
    ctx.sync()
    assert int(cnt.item()) == need, (int(cnt.item()), need)
    steps = args.join_steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    _barrier(world)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        l0 = ctx.launches()
        for i in range(steps):
            evs[i][0].record(stream)
            ctx.join_probe_async(table, dk, out, need, cnt)
            evs[i][1].record(stream)
        launches = ctx.launches() - l0
        ctx.sync()
        torch.cuda.synchronize()
    per = [a.elapsed_time(b_) for a, b_ in evs]
    ms = _max_over_ranks(float(np.mean(per)), world)
    # end to end: pinned host probe keys in, pairs out to pinned host memory
    hk = torch.from_numpy(p.keys).pin_memory()
    hout = torch.empty((need, 2), dtype=torch.int32).pin_memory()
    ctx.join_probe(table, hk, out=hout)
    e2e_steps = max(2, min(5, args.e2e_steps))
    l0 = ctx.launches()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.join_probe(table, hk, out=hout)
    e2e_s = _max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    launches += ctx.launches() - l0
    kms = _kernel_pass(ctx, min(steps, 10), lambda: ctx.join_probe_async(table, dk, out, need, cnt))
    kern_ms = kms["join_probe_ms"]
    # the kernels of one probe call, all bracketed by the events: the plan
    # (when the table has a filter or the probe is planned partitioned), the
    # Bloom pre-probe (with a filter), the partition count and scatter (when
    # planned partitioned; they return at once when the plan went direct),
    # and the probe
    pinfo = ctx.join_probe_info()
    parts = pinfo["parts"]
    planned = ctx.join_probe_partitions(table, npr)
    kernels = (["olap::join_probe_plan_kernel"] if table.has_bloom() or planned > 1 else []) + \
        (["olap::join_prefilter_kernel"] if table.has_bloom() else []) + \
        (["olap::join_part_count_kernel", "olap::join_part_scatter_kernel"] if planned > 1 else []) + \
        ["olap::join_probe_kernel"]
    peak, peak_kind = _peaks()
    m = need / npr
    honest = npr * (8 + 32) + need * 8
    stream_only = npr * 8 + need * 8
    info = table.info()
    table.free()
    return {
        "metric": "join probes/s", "unit": "Gprobes/s", "value": world * npr / (ms * 1e-3) / 1e9,
        "ms_per_step": ms, "steps": steps, "ms_median": _median_p95(per)[0], "ms_p95": _median_p95(per)[1],
        "cell": {"build_rows": nb, "build": mult, "probe_rows": npr, "dist": dist, "hit_rate": hit,
                 "pairs": need, "pairs_per_probe": m, "buckets": info["n_buckets"], "load": 0.5,
                 "rowids": "implicit", "probe_partitions": parts, "prefiltered": pinfo["prefiltered"],
                 "rows_probed_after_prefilter": pinfo["rows_probed"]},
        "build": {"ms": build_s * 1e3, "Grows_per_s": nb / build_s / 1e9},
        "roofline": {"bound": "hbm", "kernel": " + ".join(kernels), "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s",
                     "kernel_ms": kern_ms,
                     "timing": "CUDA events around the whole probe (every kernel it launches)",
                     "honest": {"bytes_per_launch": honest, "achieved": honest / (kern_ms * 1e-3) / 1e9,
                                "frac": honest / (kern_ms * 1e-3) / 1e9 / peak,
                                "bytes_per_probe": "8 key + 32 table sector + 8 per pair"},
                     "streaming_only": {"bytes_per_launch": stream_only,
                                        "achieved": stream_only / (kern_ms * 1e-3) / 1e9,
                                        "frac": stream_only / (kern_ms * 1e-3) / 1e9 / peak},
                     "traffic": args.join_traffic},
        "e2e": {"value": world * npr / e2e_s / 1e9, "unit": "Gprobes/s", "ms_per_step": e2e_s * 1e3,
                "h2d_bytes_per_step": npr * 8, "d2h_bytes_per_step": need * 8 + 8},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }


def pair_leg(args, ctx, torch, world):
    """Top-K over a two-column key, ORDER BY c0 DESC, c1 ASC LIMIT 1000, at
    2^log2n rows of two device-resident int32 columns: c0 with 1024 distinct
    values (seed 1), c1 uniform (seed 2), so ties on c0 are broken by c1.
    CUDA events around each call on the library stream; the roofline counts
    both columns read once (8 bytes per row)."""
    from paper_2601_19911_gb300 import datagen, olap
    n, k = 1 << args.log2n, args.k
    d0 = torch.from_numpy(datagen.topk_keys(n, "dup1024", "i32", seed=1)).cuda()
    d1 = torch.from_numpy(datagen.topk_keys(n, "uniform", "i32", seed=2)).cuda()
    g0 = torch.empty(k, dtype=torch.int32, device="cuda")
    g1 = torch.empty(k, dtype=torch.int32, device="cuda")
    gr = torch.empty(k, dtype=torch.int32, device="cuda")
    stream = torch.cuda.ExternalStream(ctx.stream)
    for _ in range(max(3, args.warmup)):
        ctx.topk_pair(d0, olap.DESC, d1, olap.ASC, k, out_keys0=g0, out_keys1=g1, out_rowids=gr)
    steps = max(3, min(args.steps, 100))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    _barrier(world)
    with ClockSampler(torch.cuda.current_device()) as clk:
        l0 = ctx.launches()
        for a, e in evs:
            a.record(stream)
            ctx.topk_pair(d0, olap.DESC, d1, olap.ASC, k, out_keys0=g0, out_keys1=g1, out_rowids=gr)
            e.record(stream)
        ctx.sync()
        launches = ctx.launches() - l0
    per = [a.elapsed_time(e) for a, e in evs]
    ms = _max_over_ranks(float(np.mean(per)), world)
    peak, peak_kind = _peaks()
    info = ctx.topk_info()
    del d0, d1
    torch.cuda.empty_cache()
    return {"metric": "two-column Top-K rows/s", "unit": "Grows/s", "value": world * n / (ms * 1e-3) / 1e9,
            "ms_per_step": ms, "ms_median": _median_p95(per)[0], "ms_p95": _median_p95(per)[1], "steps": steps,
            "config": {"rows": n, "k": k, "order": "c0 desc, c1 asc", "c0": "int32, 1024 distinct (seed 1)",
                       "c1": "int32 uniform (seed 2)"},
            "roofline": {"bound": "hbm", "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "bytes_per_row": 8, "achieved": n * 8 / (ms * 1e-3) / 1e9,
                         "frac": n * 8 / (ms * 1e-3) / 1e9 / peak, "timing": "CUDA events around the whole call"},
            "last_launch": info, "gpu_launches": launches, "clocks": clk.summary()}


def join_cells_leg(args, ctx, torch, world):
    """Every join cell: 2^24 build rows {unique, multiplicity 1-4} x 2^28
    probe keys {uniform, Zipf 1.1} x hit rate {0.1, 0.9}, device resident,
    seed 2 (the full-size parity tests' inputs).  Per cell: the probe call's
    time (CUDA events around every kernel it launches, mean of a few steps),
    probes/s and the fraction of the HBM roofline, with how the call ran
    (partitions, Bloom pre-probe)."""
    from paper_2601_19911_gb300 import datagen, olap
    nb, npr = 1 << args.join_log2b, 1 << args.join_log2p
    peak, peak_kind = _peaks()
    stream = torch.cuda.ExternalStream(ctx.stream)
    cells = []
    launches = 0
    with ClockSampler(torch.cuda.current_device()) as clk:
        for mult in ("unique", "mult14"):
            b = datagen.join_build(nb, mult, seed=2)
            table = ctx.join_build(torch.from_numpy(b.keys).cuda())
            for dist in ("uniform", "zipf"):
                for hit in (0.1, 0.9):
                    p = datagen.join_probe(npr, b, hit, dist, seed=2)
                    need = p.expected_pairs(b)
                    dk = torch.from_numpy(p.keys).cuda()
                    out = torch.empty((need, 2), dtype=torch.int32, device="cuda")
                    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
                    for _ in range(2):
                        ctx.join_probe_async(table, dk, out, need, cnt)
                    ctx.sync()
                    assert int(cnt.item()) == need, (mult, dist, hit, int(cnt.item()), need)
                    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                           for _ in range(args.join_cell_steps)]
                    _barrier(world)
                    l0 = ctx.launches()
                    for a, e in evs:
                        a.record(stream)
                        ctx.join_probe_async(table, dk, out, need, cnt)
                        e.record(stream)
                    ctx.sync()
                    launches += ctx.launches() - l0
                    ms = _max_over_ranks(float(np.mean([a.elapsed_time(e) for a, e in evs])), world)
                    info = ctx.join_probe_info()
                    honest = npr * (8 + 32) + need * 8
                    cells.append({"build": mult, "dist": dist, "hit_rate": hit, "pairs": need, "ms": ms,
                                  "gprobes_s": world * npr / (ms * 1e-3) / 1e9,
                                  "honest_frac": honest / (ms * 1e-3) / 1e9 / peak,
                                  "streaming_only_frac": (npr * 8 + need * 8) / (ms * 1e-3) / 1e9 / peak,
                                  "partitions": info["parts"], "prefiltered": info["prefiltered"],
                                  "rows_probed": info["rows_probed"]})
                    del dk, out
                    torch.cuda.empty_cache()
            table.free()
    return {"metric": "join probes/s per cell", "unit": "Gprobes/s", "build_rows": nb, "probe_rows": npr,
            "steps": args.join_cell_steps, "peak": peak, "peak_kind": peak_kind,
            "honest_bytes_per_probe": "8 key + 32 table sector + 8 per pair",
            "timing": "CUDA events around each probe call (every kernel it launches)", "cells": cells,
            "gpu_launches": launches, "clocks": clk.summary()}


def topk_cells_leg(args, ctx, torch, world):
    """Every Top-K-at-scale cell: 2^log2n keys in int64 and float32, uniform,
    already ascending and 1024 distinct values (seed 1), K in {10, 1000,
    100000}, DESC, explicit u32 row-ids 0..n-1, device resident (the
    full-size parity tests' inputs).  Per cell: the call's CUDA-event time
    (mean of a few calls), keys/s, the filter kernel's own time, and both
    fractions of the HBM roofline (key bytes read once)."""
    from paper_2601_19911_gb300 import datagen, olap
    n = 1 << args.log2n
    peak, peak_kind = _peaks()
    stream = torch.cuda.ExternalStream(ctx.stream)
    dr = torch.arange(n, dtype=torch.int64, device="cuda").to(torch.int32)
    cells = []
    launches = 0
    with ClockSampler(torch.cuda.current_device()) as clk:
        for kt in ("i64", "f32"):
            for dist in ("uniform", "ascending", "dup1024"):
                dk = torch.from_numpy(datagen.topk_keys(n, dist, kt, seed=1)).cuda()
                w = dk.element_size()
                for k in (10, 1000, 100_000):
                    ok = torch.empty(k, dtype=dk.dtype, device="cuda")
                    orow = torch.empty(k, dtype=torch.int32, device="cuda")
                    for _ in range(2):
                        ctx.topk_async(dk, k, olap.DESC, ok, orow, d_rowids=dr)
                    ctx.sync()
                    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                           for _ in range(args.topk_cell_steps)]
                    _barrier(world)
                    l0 = ctx.launches()
                    for a, e in evs:
                        a.record(stream)
                        ctx.topk_async(dk, k, olap.DESC, ok, orow, d_rowids=dr)
                        e.record(stream)
                    ctx.sync()
                    launches += ctx.launches() - l0
                    ms = _max_over_ranks(float(np.mean([a.elapsed_time(e) for a, e in evs])), world)
                    kms = _kernel_pass(ctx, args.topk_cell_steps,
                                       lambda: ctx.topk_async(dk, k, olap.DESC, ok, orow, d_rowids=dr))
                    info = ctx.topk_info()
                    fms = kms.get("topk_filter_ms")
                    cells.append({"key": kt, "dist": dist, "k": k, "ms": ms,
                                  "gkeys_s": world * n / (ms * 1e-3) / 1e9,
                                  "call_frac": n * w / (ms * 1e-3) / 1e9 / peak,
                                  "filter_ms": fms,
                                  "filter_frac": (n * w / (fms * 1e-3) / 1e9 / peak) if fms else None,
                                  "select_ms": kms.get("topk_select_ms"), "path": info["path"],
                                  "candidates": info["candidates"]})
                del dk, ok, orow
                torch.cuda.empty_cache()
    del dr
    torch.cuda.empty_cache()
    return {"metric": "Top-K keys/s per cell", "unit": "Gkeys/s", "n": n, "order": "desc",
            "rowids": "explicit", "steps": args.topk_cell_steps, "peak": peak, "peak_kind": peak_kind,
            "bytes_per_key": "the key width, read once",
            "timing": "CUDA events around each call on the library stream; the filter by per-kernel events",
            "cells": cells, "gpu_launches": launches, "clocks": clk.summary()}


def batched_leg(args, ctx, torch):
    """4096 Top-K queries (N ~ logU[1e3, 4e6) int64 uniform, K ~ U{1..1000},
    implicit row-ids) and 1024 probe batches (n ~ logU[1e3, 1e6)) against one
    resident 2^22-key unique table (hit rate 0.5), all device resident: one
    graph launch of the persistent executor against one library call per
    query on one stream, both on a context whose digit width, filter block
    size and load factor the autotuner picked."""
    from paper_2601_19911_gb300 import datagen, olap
    # autotuned digit width, filter block size and load factor, on a context
    # of its own: a 2^20-key Top-K (the large queries dominate the batch) and
    # the batch's table shape
    ctx = olap.Context(torch.cuda.current_device(), batch_overlap=args.batch_overlap,
                       batch_topk_ctas_per_sm=args.batch_topk_ctas)
    tune = ctx.autotune(topk_n=1 << 20, topk_k=500, join_build_n=1 << 22, join_probe_n=1 << 20,
                        join_hit_rate=0.5, reps=5)
    ns, ks = datagen.batched_topk_queries(args.batch_topk, 1e3, 4e6, 1000, seed=3)
    offs = np.concatenate([[0], np.cumsum(ns)])
    keys = datagen.splitmix64_torch(datagen.stream_seed(3, 0), int(offs[-1]), device="cuda")
    koffs = np.concatenate([[0], np.cumsum(ks)])
    out_k = torch.empty(int(koffs[-1]), dtype=torch.int64, device="cuda")
    out_r = torch.empty(int(koffs[-1]), dtype=torch.int32, device="cuda")
    nitems = args.batch_topk + args.batch_probe
    counts = torch.zeros(nitems, dtype=torch.int64, device="cuda")
    status = torch.zeros(nitems, dtype=torch.int32, device="cuda")
    items = []
    for i in range(args.batch_topk):
        items.append(olap.topk_item(keys[int(offs[i]):int(offs[i + 1])], int(ks[i]), olap.DESC,
                                    out_k[int(koffs[i]):int(koffs[i + 1])], out_r[int(koffs[i]):int(koffs[i + 1])],
                                    counts[i:i + 1], d_status=status[i:i + 1]))
    b = datagen.join_build(1 << 22, "unique", seed=3)
    table = ctx.join_build(torch.from_numpy(b.keys).cuda())
    pns = datagen.batched_probe_sizes(args.batch_probe, 1e3, 1e6, seed=3)
    poffs = np.concatenate([[0], np.cumsum(pns)])
    p = datagen.join_probe(int(poffs[-1]), b, 0.5, "uniform", seed=3)
    hits = np.concatenate([[0], np.cumsum(p.hit)])
    pk = torch.from_numpy(p.keys).cuda()
    pairs = torch.empty((int(hits[-1]) + 1, 2), dtype=torch.int32, device="cuda")
    for j in range(args.batch_probe):
        a, e = int(poffs[j]), int(poffs[j + 1])
        h0, h1 = int(hits[a]), int(hits[e])
        items.append(olap.probe_item(table, pk[a:e], pairs[h0:h1 + 1], h1 - h0,
                                     counts[args.batch_topk + j:args.batch_topk + j + 1],
                                     d_status=status[args.batch_topk + j:args.batch_topk + j + 1]))
    batch = ctx.batch(items)
    stream = torch.cuda.ExternalStream(ctx.stream)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        ctx.sync()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ctx.launches()
        a_.record(stream)
        for _ in range(reps):
            fn()
        b_.record(stream)
        n_launch = ctx.launches() - l0
        ctx.sync()
        torch.cuda.synchronize()
        return a_.elapsed_time(b_) / reps, n_launch

    with ClockSampler(torch.cuda.current_device()) as clk:
        ms_graph, launch_graph = timed(batch.run, args.batch_reps)
    errors = batch.errors()
    ok = int((status != olap.OK).sum().item()) == 0
    ms_per_query, launch_pq = timed(batch.run_per_query, max(1, args.batch_reps // 5))
    peak, peak_kind = _peaks()
    algo = float(offs[-1]) * 8 + float(ks.sum()) * 24 + float(poffs[-1]) * 40 + float(hits[-1]) * 8
    batch.free()
    table.free()
    ctx.close()
    return {"metric": "batched vs per-query speedup", "value": ms_per_query / ms_graph, "unit": "x",
            "graph_ms": ms_graph, "per_query_ms": ms_per_query, "device_errors": errors, "all_ok": ok,
            "items": {"topk": args.batch_topk, "probe": args.batch_probe, "topk_keys": int(offs[-1]),
                      "probes": int(poffs[-1]), "pairs": int(hits[-1])},
            "roofline": {"bound": "hbm", "algorithmic_bytes": algo, "achieved": algo / (ms_graph * 1e-3) / 1e9,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": algo / (ms_graph * 1e-3) / 1e9 / peak,
                         "bytes": "8 per Top-K key + 24 per selected row + 40 per probe + 8 per pair"},
            "gpu_launches": launch_graph + launch_pq,
            "gpu_launches_per_graph_run": launch_graph // args.batch_reps,
            "gpu_launches_per_query_run": launch_pq // max(1, args.batch_reps // 5),
            "autotune": tune, "clocks": clk.summary()}


def _median_ms(fn, reps=3):
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        ts.append((time.perf_counter() - t0) * 1e3)
    return float(np.median(ts))


def fullrow_leg(args, ctx, torch):
    """Full-row vs key-only transfer with late materialization (Sec. V-E, the
    Stage-1 proxy; Sec. II-C).  A table of N rows, each a float64 key (the
    paper's `value double`) followed by a payload of `--fullrow-payload`
    bytes, in pinned host memory, and its key column (a columnar engine's
    key-only source).  ORDER BY key DESC LIMIT 100:
      * full row: olap_topk_rows moves the whole rows H2D, extracts the keys,
        selects and returns the 100 rows whole;
      * key only: olap_topk moves only the key column (row-ids implicit) and
        returns 100 row-ids; the host then gathers those 100 rows (late
        materialization).
    Also the H2D copy alone of each (the transfer term), and the host cost of
    cutting the key column out of the row table for a row store.  Medians."""
    from paper_2601_19911_gb300 import datagen, olap
    P = args.fullrow_payload
    rb = 8 + P
    host = olap.HostEngine(threads=args.host_threads)
    kk = 100
    reps = args.fullrow_reps
    out = {}
    for n in (3_000_000, 1 << 24):
        keys = datagen.topk_keys(n, "uniform", "f64", seed=7)
        rows = torch.empty((n, rb), dtype=torch.uint8).pin_memory()
        rn = rows.numpy()
        rn[:, 8:] = np.frombuffer(datagen.splitmix64(8, (n * P + 7) // 8).tobytes(), dtype=np.uint8)[: n * P] \
            .reshape(n, P)
        rn[:, :8] = keys.view(np.uint8).reshape(n, 8)
        kcol = torch.from_numpy(keys).pin_memory()
        orows = torch.empty(kk * rb, dtype=torch.uint8).pin_memory()
        orid = torch.empty(kk, dtype=torch.int32).pin_memory()
        okeys = torch.empty(kk, dtype=torch.float64).pin_memory()
        dev_rows = torch.empty((n, rb), dtype=torch.uint8, device="cuda")
        dev_keys = torch.empty(n, dtype=torch.float64, device="cuda")

        def full():
            ctx.topk_rows(rows, rb, 0, olap.KEY_F64, kk, olap.DESC, out_rows=orows, out_rowids=orid)

        def key_only():
            _, rid = ctx.topk(kcol, kk, olap.DESC, out_keys=okeys, out_rowids=orid)
            return rn[rid.numpy().view(np.uint32)]                  # late materialization on the host

        def tx_rows():
            dev_rows.copy_(rows, non_blocking=True)
            torch.cuda.synchronize()

        def tx_keys():
            dev_keys.copy_(kcol, non_blocking=True)
            torch.cuda.synchronize()

        def extract():
            host.extract(rn, rb, 0, np.float64)

        got = key_only()
        full()
        assert np.array_equal(got.reshape(-1), orows.numpy()[: kk * rb])   # same rows either way
        t = {nm: _median_ms(fn, reps) for nm, fn in (("full_row_e2e", full), ("key_only_e2e", key_only),
                                                     ("full_row_transfer", tx_rows),
                                                     ("key_only_transfer", tx_keys),
                                                     ("row_store_key_extraction", extract))}
        out[f"n{n}"] = {**{k: round(v, 4) for k, v in t.items()},
                        "transfer_reduction": t["full_row_transfer"] / t["key_only_transfer"],
                        "e2e_speedup": t["full_row_e2e"] / t["key_only_e2e"],
                        "e2e_speedup_row_store": t["full_row_e2e"] / (t["key_only_e2e"] +
                                                                      t["row_store_key_extraction"]),
                        "bytes_full_row": n * rb, "bytes_key_only": n * 8}
        del rows, kcol, dev_rows, dev_keys
        torch.cuda.empty_cache()
    host.close()
    return {"metric": "full-row vs key-only + late materialization (Top-100, float64 key)",
            "host_threads": args.serve_cpu_workers,
            "payload_bytes": P, "row_bytes": rb, "reps": reps, "unit": "ms (medians) and ratios", **out}


def _crossover(ns, gain):
    """Smallest N where the measured gain (ms) turns positive and stays so,
    interpolated in log N between the two grid points around the sign change;
    0 if it never turns positive, ns[0] if it is positive everywhere."""
    pos = [g > 0.0 for g in gain]
    if all(pos):
        return float(ns[0])
    if not pos[-1]:
        return 0.0
    i = max(j for j in range(len(pos)) if not pos[j])
    g0, g1 = gain[i], gain[i + 1]
    x0, x1 = np.log(ns[i]), np.log(ns[i + 1])
    return float(np.exp(x0 + (x1 - x0) * (-g0) / (g1 - g0)))


def gate_leg(args, ctx, torch):
    """Risky Gate validation (Sec. V-D break-even, Sec. IV gate margin):
    Top-K (K = 100, int64) and probe (against a resident 2^22-key table, hit
    rate 0.9) over a log-spaced N grid from 1e3 to 1e8, keys in pageable host
    memory.  At each N the host engine's time and the GPU path's end-to-end
    time (key-only transfer, kernel, result return) are measured; the gate is
    calibrated from the odd grid points (measured component times, 1/y^2
    weights); its break-even N* for margins 0, 5 and 10 ms is compared with
    the measured crossover (interpolated in log N over the whole grid), and
    the offload decision at every grid point is reported per margin."""
    from paper_2601_19911_gb300 import datagen, olap
    ns = np.unique(np.floor(np.logspace(3, 8, args.gate_points)).astype(np.int64))
    A = int(ns[-1])
    host = olap.HostEngine(threads=args.host_threads)
    arena = datagen.topk_keys(A, "uniform", "i64", seed=5)
    b = datagen.join_build(1 << 22, "unique", seed=5)
    table = ctx.join_build(b.keys)
    host.add_table(b.keys)
    p = datagen.join_probe(A, b, 0.9, "uniform", seed=5)
    cum = np.concatenate([[0], np.cumsum(p.hit)])
    dev = torch.from_numpy(arena).cuda()
    kk = 100
    rows = {olap.OP_TOPK: [], olap.OP_PROBE: []}
    for n in (int(x) for x in ns):
        keys = arena[:n]
        ok = np.empty(kk, dtype=np.int64)
        orow = np.empty(kk, dtype=np.uint32)
        req = olap.olap_serve_request(olap.OP_TOPK, olap.KEY_I64, olap.DESC, 0, keys.ctypes.data, None, n, kk,
                                      None, 0.0, 0.0, ok.ctypes.data, orow.ctypes.data, None, 0)
        t_cpu = _median_ms(lambda: host.run(req), args.gate_reps)
        dok = torch.empty(kk, dtype=torch.int64, device="cuda")
        dor = torch.empty(kk, dtype=torch.int32, device="cuda")
        t_in = _median_ms(lambda: ctx.topk(keys, kk, olap.DESC, out_keys=dok, out_rowids=dor), args.gate_reps)
        t_all = _median_ms(lambda: ctx.topk(keys, kk, olap.DESC, out_keys=ok, out_rowids=orow), args.gate_reps)

        def kern():
            ctx.topk_async(dev[:n], kk, olap.DESC, dok, dor)
            ctx.sync()
        t_ker = _median_ms(kern, args.gate_reps)
        # transfer and post-processing as signed differences of the measured
        # calls, so that the three terms add up to the end-to-end time
        rows[olap.OP_TOPK].append((n, kk, 8.0 * n, min(kk, n), t_cpu, t_in - t_ker, t_ker, t_all - t_in, t_all))
        pk = p.keys[:n]
        need = int(cum[n])
        out = np.empty((need + 64, 2), dtype=np.uint32)
        preq = olap.olap_serve_request(olap.OP_PROBE, olap.KEY_I64, 0, 0, pk.ctypes.data, None, n, 0,
                                       table.h.value, float(need), 0.0, None, None, out.ctypes.data, need + 64)
        t_cpu = _median_ms(lambda: host.run(preq), args.gate_reps)
        dout = torch.empty((need + 64, 2), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        t_in = _median_ms(lambda: ctx.join_probe(table, pk, out=dout), args.gate_reps)
        t_all = _median_ms(lambda: ctx.join_probe(table, pk, out=out), args.gate_reps)
        dpk = torch.from_numpy(pk).cuda()

        def pkern():
            ctx.join_probe_async(table, dpk, dout, need + 64, cnt)
            ctx.sync()
        t_ker = _median_ms(pkern, args.gate_reps)
        del dpk
        rows[olap.OP_PROBE].append((n, 1.0 + need / n, 8.0 * n, need, t_cpu, t_in - t_ker, t_ker, t_all - t_in,
                                    t_all))
    del dev
    table.free()
    host_split = {op: host.parallel_from(op) for op in (olap.OP_TOPK, olap.OP_PROBE)}
    host.close()
    torch.cuda.empty_cache()
    result = {}
    for op, name in ((olap.OP_TOPK, "topk_k100"), (olap.OP_PROBE, "probe_hit0.9")):
        r = rows[op]
        cal = r[1::2]                                          # calibration points
        gn = [x[0] for x in r]
        mpp = r[-1][3] / r[-1][0]                              # pairs per probe

        split = float(host_split[op])

        def fit(points, margin, cpu_split):
            m = olap.gate_calibrate(op, *list(zip(*[x[:8] for x in points])), margin_ms=margin,
                                    weighting=olap.FIT_RELATIVE, cpu_split_n=cpu_split)
            if op == olap.OP_TOPK:
                return m, olap.gate_estimate(m, op, 1 << 20, kk, 8.0 * (1 << 20), kk, 8.0).n_star
            return m, olap.gate_estimate(m, op, 1 << 20, 1.0 + mpp, 8.0 * (1 << 20), mpp * (1 << 20), 8.0,
                                         mpp).n_star

        per_margin = {}
        for margin in (0.0, 5.0, 10.0):
            # the CPU cost per regime of the host engine (serial below the
            # size it goes parallel at, parallel above), and one fit over
            # everything for comparison
            _, nstar_one = fit(cal, margin, 0.0)
            m, nstar = fit(cal, margin, split)
            if op == olap.OP_TOPK:
                dec = [bool(olap.gate_estimate(m, op, x[0], kk, x[2], x[3], 8.0).offload) for x in r]
            else:
                dec = [bool(olap.gate_estimate(m, op, x[0], x[1], x[2], x[3], 8.0, mpp).offload) for x in r]
            measured = _crossover(gn, [x[4] - x[8] - margin for x in r])
            per_margin[f"{margin:g}ms"] = {
                "n_star_predicted": int(nstar), "crossover_measured": measured,
                "rel_error": (abs(nstar - measured) / measured) if measured > 0 and nstar > 0 else None,
                "n_star_one_regime_fit": int(nstar_one),
                "rel_error_one_regime_fit": (abs(nstar_one - measured) / measured)
                if measured > 0 and nstar_one > 0 else None,
                "offload_at_n": dec}
        result[name] = {"cpu_split_n": split, "n": gn, "t_host_ms": [x[4] for x in r],
                        "t_gpu_e2e_ms": [x[8] for x in r],
                        "t_tx_ms": [x[5] for x in r], "t_kernel_ms": [x[6] for x in r],
                        "t_post_ms": [x[7] for x in r], "margins": per_margin}
    return {"metric": "gate break-even: predicted N* vs measured crossover", "unit": "relative error",
            "grid_points": len(ns),
            "calibration": "odd grid points, 1/y^2-weighted least squares, the CPU cost fitted per regime of the "
                           "host engine (below and above the size it goes parallel at); transfer and "
                           "post-processing as signed differences of the measured calls",
            "reps": args.gate_reps, "host_threads": args.host_threads, **result}


def serving_leg(args, ctx, torch):
    """The serving stream: Poisson arrivals, half Top-K (N ~ logU[1e3, 1e8),
    K ~ logU[1, 1e5) clipped to N), half probes (n ~ logU[1e3, 1e8)) against
    8 resident tables of logU[1M, 16M) unique keys with hit rate 10% or 90%,
    keys sliced at seeded offsets from host column arenas and staged through
    pinned double buffers.  The gate is calibrated from measured host-engine,
    transfer, kernel and result times; the arrival rate is 0.7 x the
    always-on closed-loop throughput; gated and always-on serve the same
    trace."""
    from paper_2601_19911_gb300 import datagen, olap
    A = args.serve_arena
    rng = np.random.default_rng(4)
    topk_arena = datagen.topk_keys(A, "uniform", "i64", seed=4)
    D = datagen.join_build(1 << 24, "unique", seed=4)
    # with --serve-pin the host engine computes on the last serve_cpu_workers
    # host cores and the serving loop's own threads (GPU slots, staging
    # copies) start on the others
    cpus_all = sorted(os.sched_getaffinity(0))
    w = args.serve_cpu_workers
    pin = bool(args.serve_pin) and len(cpus_all) > w
    host_cpus = cpus_all[-w:] if pin else None
    gpu_cpus = cpus_all[:-w] if pin else None
    host = olap.HostEngine(threads=w, cpus=host_cpus)
    sizes = np.sort(datagen.log_uniform(1 << 20, 1 << 24, datagen.stream_seed(4, 12), 8))
    tables, tbytes = [], 0
    for t in range(8):
        keys_t = D.keys[: int(sizes[t])]
        tables.append(ctx.join_build(keys_t))
        host.add_table(keys_t)
        tbytes += int(sizes[t]) * 32 // 1
    common = datagen.JoinBuild(D.keys[: 1 << 20], D.keys[: 1 << 20], np.ones(1 << 20, dtype=np.int64))
    arenas = []
    for j, hit in enumerate((0.1, 0.9)):
        p = datagen.join_probe(A, common, hit, "uniform", seed=40 + j)
        arenas.append((hit, p.keys, np.concatenate([[0], np.cumsum(p.hit)])))

    # Long streams write their results into a ring of output buffers shared
    # by requests i, i + R, ... (their contents are not checked; per-request
    # buffers for 10^5 requests would take terabytes).
    ring = args.serve_requests > 5000
    R = 8
    ring_topk = [(np.empty(100_000, dtype=np.int64), np.empty(100_000, dtype=np.uint32)) for _ in range(R)] \
        if ring else None
    ring_probe = [np.empty((A + 64, 2), dtype=np.uint32) for _ in range(R)] if ring else None

    def make_requests(count, seed):
        r_ = np.random.default_rng(seed)
        reqs, keep = [], []
        for i in range(count):
            n = int(min(A, np.floor(1e3 * (1e8 / 1e3) ** r_.random())))
            off = int(r_.integers(0, A - n + 1))
            if i % 2 == 0:
                k = int(min(n, np.floor(1e5 ** r_.random())))
                if ring:
                    ok, orow = ring_topk[(i // 2) % R]
                else:
                    ok = np.empty(max(1, k), dtype=np.int64)
                    orow = np.empty(max(1, k), dtype=np.uint32)
                keys = topk_arena[off:off + n]
                keep.append((ok, orow))
                reqs.append(olap.olap_serve_request(olap.OP_TOPK, olap.KEY_I64, olap.DESC, 0, keys.ctypes.data, None,
                                                    n, k, None, 0.0, 0.0, ok.ctypes.data, orow.ctypes.data, None, 0))
            else:
                t = int(r_.integers(0, 8))
                hit, pk, cum = arenas[int(r_.integers(0, 2))]
                need = int(cum[off + n] - cum[off])
                out = ring_probe[(i // 2) % R] if ring else np.empty((need + 64, 2), dtype=np.uint32)
                keep.append((out,))
                reqs.append(olap.olap_serve_request(olap.OP_PROBE, olap.KEY_I64, 0, t, pk[off:off + n].ctypes.data,
                                                    None, n, 0, tables[t].h.value, float(need), 0.0, None, None,
                                                    out.ctypes.data, need + 64))
        return (olap.olap_serve_request * count)(*reqs), keep

    # -- gate calibration from measured times (one request at a time), on a
    # context with the same host path as the serving slots --------------------
    hacc = olap.HOST_STAGED if args.serve_host == "staged" else olap.HOST_AUTO
    sctx = olap.Context(torch.cuda.current_device(), host_access=hacc)
    cal_n = np.unique(np.floor(np.logspace(3, 8, args.serve_cal_points)).astype(np.int64))
    cal_n = cal_n[cal_n <= A]
    samples = {olap.OP_TOPK: [], olap.OP_PROBE: []}
    # K varies over the calibration points (the stream's K spans 1..1e5), so
    # the fit can tell the N*K and N*log N forms apart
    k_cycle = [10, 1000, 100000, 1, 100, 10000]
    dev_keys = torch.from_numpy(topk_arena).cuda()
    for ci, n in enumerate(cal_n):
        n = int(n)
        kcal = min(k_cycle[ci % len(k_cycle)], n)
        keys = topk_arena[:n]
        ok = np.empty(kcal, dtype=np.int64)
        orow = np.empty(kcal, dtype=np.uint32)
        req = olap.olap_serve_request(olap.OP_TOPK, olap.KEY_I64, olap.DESC, 0, keys.ctypes.data, None, n, kcal,
                                      None, 0.0, 0.0, ok.ctypes.data, orow.ctypes.data, None, 0)
        t_cpu = _median_ms(lambda: host.run(req))
        dok = torch.empty(kcal, dtype=torch.int64, device="cuda")
        dor = torch.empty(kcal, dtype=torch.int32, device="cuda")
        t_in = _median_ms(lambda: sctx.topk(keys, kcal, olap.DESC, out_keys=dok, out_rowids=dor))
        t_all = _median_ms(lambda: sctx.topk(keys, kcal, olap.DESC))
        def kern():
            sctx.topk_async(dev_keys[:n], kcal, olap.DESC, dok, dor)
            sctx.sync()
        t_ker = _median_ms(kern)
        samples[olap.OP_TOPK].append((n, kcal, 8.0 * n, min(kcal, n), t_cpu, t_in - t_ker, t_ker, t_all - t_in))
        hit, pk, cum = arenas[1]
        pkeys = pk[:n]
        need = int(cum[n])
        out = np.empty((need + 64, 2), dtype=np.uint32)
        preq = olap.olap_serve_request(olap.OP_PROBE, olap.KEY_I64, 0, 0, pkeys.ctypes.data, None, n, 0,
                                       tables[0].h.value, float(need), 0.0, None, None, out.ctypes.data, need + 64)
        t_cpu = _median_ms(lambda: host.run(preq))
        dpk = dev_keys  # reuse the device buffer for the probe keys
        dpk[:n].copy_(torch.from_numpy(pkeys))
        dout = torch.empty((need + 64, 2), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        t_in = _median_ms(lambda: sctx.join_probe(tables[0], pkeys, out=dout))
        t_all = _median_ms(lambda: sctx.join_probe(tables[0], pkeys, out=out))
        def pkern():
            sctx.join_probe_async(tables[0], dpk[:n], dout, need + 64, cnt)
            sctx.sync()
        t_ker = _median_ms(pkern)
        samples[olap.OP_PROBE].append((n, 1.0 + need / n, 8.0 * n, need, t_cpu, t_in - t_ker, t_ker,
                                       t_all - t_in))
        dev_keys[:n].copy_(torch.from_numpy(keys))
    del dev_keys
    torch.cuda.empty_cache()
    models = {}
    for op, rows in samples.items():
        cols = list(zip(*rows))
        models[op] = olap.gate_calibrate(op, *cols, margin_ms=args.serve_margin, weighting=olap.FIT_RELATIVE,
                                         topk_cpu=olap.CPU_MAX if args.serve_topk_cpu == "max" else 0,
                                         cpu_split_n=float(host.parallel_from(op)))
    # -- arrival rate from the closed-loop always-on throughput -----------------
    reqs, keep = make_requests(args.serve_requests, seed=4)
    budget = max(1, args.serve_budget_gb * (1 << 30) - tbytes)
    # closed-loop throughput on the first (at most 2000) requests of the trace
    cl_reqs, _cl_keep = make_requests(min(args.serve_requests, 2000), seed=4)
    if pin:
        os.sched_setaffinity(0, gpu_cpus)      # the threads olap.serve starts inherit it
    closed = olap.serve(cl_reqs, olap.SERVE_ALWAYS_GPU, gpu_slots=args.serve_slots, mem_budget_bytes=budget,
                        closed_loop=True, host_access=hacc)
    lam = 0.7 * closed.throughput_rps
    arrivals = datagen.poisson_arrivals(args.serve_requests, lam, seed=4) * 1e3
    out = {}
    for name, policy in (("always_on", olap.SERVE_ALWAYS_GPU), ("gated", olap.SERVE_GATED)):
        for i in range(args.serve_requests):
            reqs[i].arrival_ms = float(arrivals[i])
        st = olap.serve(reqs, policy, models[olap.OP_TOPK], models[olap.OP_PROBE], host,
                        gpu_slots=args.serve_slots, cpu_workers=args.serve_cpu_workers, mem_budget_bytes=budget,
                        host_access=hacc)
        out[name] = {"p50_ms": st.p50_ms, "p95_ms": st.p95_ms, "p99_ms": st.p99_ms, "mean_ms": st.mean_ms,
                     "max_ms": st.max_ms, "throughput_rps": st.throughput_rps, "wall_ms": st.wall_ms,
                     "offload_fraction": st.offload_fraction, "n_gpu": st.n_gpu, "n_host": st.n_host,
                     "failed": st.n_failed, "peak_reserved_gb": st.peak_reserved_bytes / 2**30}
    if pin:
        os.sched_setaffinity(0, cpus_all)
    def mdict(m):
        return {"cpu_form": ["n_log2_n", "n_k", "n_m", "max(n_log2_n, n_k)"][m.cpu_form], "a": m.a, "b": m.b,
                "a2": m.a2, "b2": m.b2, "c_ms_per_byte": m.c,
                "d": m.d, "e": m.e, "f": m.f, "g": m.g, "h": m.h, "margin_ms": m.margin_ms}
    nstar = olap.gate_estimate(models[olap.OP_TOPK], olap.OP_TOPK, 1 << 20, 100, 8.0 * (1 << 20), 100, 8.0).n_star
    for t in tables:
        t.free()
    host.close()
    hdirect = sctx.host_direct
    sctx.close()
    return {"metric": "gated vs always-on P99 latency (ms)", "value": out["gated"]["p99_ms"], "unit": "ms",
            "higher_is_better": False, "requests": args.serve_requests, "arrival_rate_rps": lam,
            "closed_loop_always_on_rps": closed.throughput_rps, "gpu_slots": args.serve_slots,
            "budget_gb": args.serve_budget_gb, "arena_keys": A, "tables": [int(x) for x in sizes],
            "host_path": "direct device access" if hdirect else "pinned staging",
            "host_engine": {"workers": w, "cores": host_cpus or "any", "serving_threads_cores": gpu_cpus or "any"},
            "gated": out["gated"], "always_on": out["always_on"],
            "gate": {"topk": mdict(models[olap.OP_TOPK]), "probe": mdict(models[olap.OP_PROBE]),
                     "topk_n_star_k100": int(nstar), "calibration_points": len(cal_n)}}


def _median_p95(xs):
    """Median and 95th percentile (linear interpolation) of a list of times."""
    a = np.asarray(xs, dtype=np.float64)
    return float(np.median(a)), float(np.percentile(a, 95))


def single_leg(args, ctx, torch):
    """The single Top-K query: 2^20 int64 keys drawn uniformly over the full
    range (seed 0), explicit row-ids 0..N-1, K = 100, DESC.  The keys fit in
    L2, so this is a latency figure: one query at a time, 31 warmed runs,
    median and P95, kernel-only (device-resident keys and row-ids, CUDA
    events around each call) and end to end through the blocking call (keys
    and row-ids, 12 MiB, from pinned host memory, and again from pageable
    host memory; K results back to the same kind of memory)."""
    from paper_2601_19911_gb300 import datagen, olap
    n, k, reps = 1 << 20, 100, 31
    keys = datagen.topk_keys(n, "uniform", "i64", seed=0)
    rid = datagen.identity_rowids(n)
    dk = torch.from_numpy(keys).cuda()
    dr = torch.from_numpy(rid.view(np.int32)).cuda()
    ok = torch.empty(k, dtype=torch.int64, device="cuda")
    orow = torch.empty(k, dtype=torch.int32, device="cuda")
    stream = torch.cuda.ExternalStream(ctx.stream)
    for _ in range(5):
        ctx.topk_async(dk, k, olap.DESC, ok, orow, d_rowids=dr)
    ctx.sync()
    kern = []
    l0 = ctx.launches()
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.topk_async(dk, k, olap.DESC, ok, orow, d_rowids=dr)
        b.record(stream)
        ctx.sync()
        kern.append(a.elapsed_time(b))
    launches = ctx.launches() - l0

    def e2e(kk, rr, o1, o2):
        nonlocal launches
        for _ in range(3):
            ctx.topk(kk, k, olap.DESC, rowids=rr, out_keys=o1, out_rowids=o2)
        ts = []
        c0 = ctx.launches()
        for _ in range(reps):
            t0 = time.perf_counter()
            ctx.topk(kk, k, olap.DESC, rowids=rr, out_keys=o1, out_rowids=o2)
            ts.append((time.perf_counter() - t0) * 1e3)
        launches += ctx.launches() - c0
        return ts

    pinned = e2e(torch.from_numpy(keys).pin_memory(), torch.from_numpy(rid.view(np.int32)).pin_memory(),
                 torch.empty(k, dtype=torch.int64).pin_memory(), torch.empty(k, dtype=torch.int32).pin_memory())
    pageable = e2e(keys, rid, np.empty(k, dtype=np.int64), np.empty(k, dtype=np.uint32))
    km, kp = _median_p95(kern)
    pm, pp = _median_p95(pinned)
    gm, gp = _median_p95(pageable)
    return {"metric": "single Top-K query latency", "unit": "ms (median, p95 of 31)",
            "config": {"n": n, "k": k, "order": "desc", "key_type": "i64", "rowids": "explicit", "seed": 0},
            "kernel": {"median_ms": km, "p95_ms": kp, "gkeys_s": n / (km * 1e-3) / 1e9},
            "e2e_pinned": {"median_ms": pm, "p95_ms": pp, "gkeys_s": n / (pm * 1e-3) / 1e9,
                           "h2d_bytes": n * 12, "d2h_bytes": k * 12},
            "e2e_pageable": {"median_ms": gm, "p95_ms": gp, "gkeys_s": n / (gm * 1e-3) / 1e9,
                             "host_access": "direct" if ctx.host_direct else "staged"},
            "gpu_launches": launches}


def link_leg(torch, nbytes: int = 1 << 30, reps: int = 10):
    """The host link every offload crosses: pinned host <-> device copy
    bandwidth (cudaMemcpyAsync through torch) of `nbytes`, CUDA events,
    median of `reps`."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()

    def rate(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return nbytes / (float(np.median(ts)) * 1e-3) / 1e9

    h2d = rate(lambda: d.copy_(h, non_blocking=True))
    d2h = rate(lambda: h.copy_(d, non_blocking=True))
    del h, d
    torch.cuda.empty_cache()
    return {"h2d_gbs": h2d, "d2h_gbs": d2h, "bytes": nbytes, "reps": reps,
            "memory": "pinned host <-> device, cudaMemcpyAsync"}


def _parse_cpu_model(lscpu: str, cpuinfo: str):
    """CPU model name from `lscpu` output ("Model name:"), else from
    /proc/cpuinfo ("model name"), else None."""
    for text, key in ((lscpu, "model name:"), (cpuinfo, "model name")):
        for ln in text.splitlines():
            if ln.strip().lower().startswith(key):
                v = ln.split(":", 1)[1].strip() if ":" in ln else ""
                if v and v != "-":
                    return v
    return None


def _host_info():
    """Cores and CPU model of the machine the CPU baseline runs on."""
    import platform
    lscpu = cpuinfo = ""
    try:
        lscpu = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            cpuinfo = f.read()
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "machine": platform.machine(),
            "cpu_model": _parse_cpu_model(lscpu, cpuinfo)}


def _gpu_cpu_affinity(index: int):
    """CPU cores local to GPU `index` from `nvidia-smi topo -m` (its "CPU
    Affinity" column), as a set, or None when unknown."""
    import subprocess
    try:
        out = subprocess.run(["nvidia-smi", "topo", "-m"], capture_output=True, text=True, timeout=30).stdout
    except Exception:
        return None
    return _parse_topo_affinity(out, index)


def _parse_topo_affinity(out: str, index: int):
    """The "CPU Affinity" cell of row GPU`index` in `nvidia-smi topo -m`
    output (tab-separated; ranges like "0-71,144-215") as a set of core
    numbers, or None when the table, the row or the column is missing."""
    lines = [ln for ln in out.splitlines() if ln.strip()]
    if not lines:
        return None
    head = lines[0].split("\t")
    col = next((i for i, h in enumerate(head) if "CPU Affinity" in h), None)
    row = next((ln for ln in lines[1:] if ln.split("\t")[0].strip() == f"GPU{index}"), None)
    if col is None or row is None:
        return None
    fields = row.split("\t")
    if col >= len(fields):
        return None
    cpus = set()
    try:
        for part in fields[col].strip().split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
    except ValueError:
        return None
    return cpus or None


def _bind_near_gpu(index: int):
    """Run this process on the cores of the GPU's own socket, so host buffers
    (first-touch) sit next to its NVLink-C2C link; returns the binding made."""
    cpus = _gpu_cpu_affinity(index)
    if not cpus:
        return None
    try:
        os.sched_setaffinity(0, cpus & os.sched_getaffinity(0) or cpus)
    except OSError:
        return None
    got = sorted(os.sched_getaffinity(0))
    return f"{got[0]}-{got[-1]} ({len(got)} cores)"


def run_ours(args):
    import torch
    world, rank, local = _dist()
    affinity = _bind_near_gpu(local if world > 1 else 0)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2601_19911_gb300 import datagen, olap

    n, k = 1 << args.log2n, args.k
    workloads = args.workload.split(",")
    filt = {"bulk": olap.FILTER_BULK, "regs": olap.FILTER_REGS}[args.filter]
    ctx = olap.Context(torch.cuda.current_device(), topk_filter=filt, topk_tile_bytes=args.tile,
                       topk_stages=args.stages, topk_ctas_per_sm=args.ctas_per_sm,
                       join_partitions=args.join_partitions, join_bucket_loads=args.join_loads,
                       l2_fetch_bytes=args.l2_fetch)
    keys = datagen.topk_keys(n, args.dist, args.key_type, seed=1)
    w = keys.dtype.itemsize
    dk = torch.from_numpy(keys).cuda()
    rid_host = datagen.identity_rowids(n) if args.rowids == "explicit" else None
    dr = None if rid_host is None else torch.from_numpy(rid_host.view(np.int32)).cuda()
    ok = torch.empty(k, dtype=dk.dtype, device="cuda")
    orow = torch.empty(k, dtype=torch.int32, device="cuda")
    stream = torch.cuda.ExternalStream(ctx.stream)

    # -- kernel-only: device-resident keys, one launch per step ----------------
    for _ in range(max(3, args.warmup)):
        ctx.topk_async(dk, k, olap.DESC, ok, orow, d_rowids=dr)
    ctx.sync()
    _barrier(world)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        l0 = ctx.launches()
        start.record(stream)
        for i in range(args.steps):
            evs[i][0].record(stream)
            ctx.topk_async(dk, k, olap.DESC, ok, orow, d_rowids=dr)
            evs[i][1].record(stream)
        end.record(stream)
        launches = ctx.launches() - l0
        ctx.sync()
        torch.cuda.synchronize()
    total_ms = start.elapsed_time(end)
    per_launch = [a.elapsed_time(b) for a, b in evs]
    phases = ctx.topk_info()
    total_ms = _max_over_ranks(total_ms, world)
    ms = total_ms / args.steps
    from paper_2601_19911_gb300 import replicas
    value = replicas.whole_job_rate(n, world, ms * 1e-3) / 1e9

    # -- end to end through the public blocking call, pinned host keys -----------
    hk = torch.from_numpy(keys).pin_memory()
    hr = None if rid_host is None else torch.from_numpy(rid_host.view(np.int32)).pin_memory()
    hok = torch.empty(k, dtype=dk.dtype).pin_memory()
    horow = torch.empty(k, dtype=torch.int32).pin_memory()
    for _ in range(2):
        ctx.topk(hk, k, olap.DESC, rowids=hr, out_keys=hok, out_rowids=horow)
    _barrier(world)
    e2e_steps = max(3, min(args.steps, args.e2e_steps))
    l0 = ctx.launches()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.topk(hk, k, olap.DESC, rowids=hr, out_keys=hok, out_rowids=horow)
    e2e_s = _max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    launches += ctx.launches() - l0
    e2e_value = replicas.whole_job_rate(n, world, e2e_s) / 1e9
    e2e_info = ctx.topk_info()
    # on the sampled path pinned row-ids stay in host memory: the kernels
    # read the candidates' row-ids there, and only the keys are copied
    rid_in_place = hr is not None and e2e_info["rowids_in_place"]
    e2e_keys_only = None
    if hr is not None:
        # the same call with implicit row-ids: only the keys cross the link
        ctx.topk(hk, k, olap.DESC, out_keys=hok, out_rowids=horow)
        _barrier(world)
        l0 = ctx.launches()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            ctx.topk(hk, k, olap.DESC, out_keys=hok, out_rowids=horow)
        ko_s = _max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
        launches += ctx.launches() - l0
        e2e_keys_only = {"value": replicas.whole_job_rate(n, world, ko_s) / 1e9, "unit": "Gkeys/s",
                         "h2d_bytes_per_step": n * w, "d2h_bytes_per_step": k * (w + 4) + 4,
                         "ms_per_step": ko_s * 1e3}

    # -- per-kernel device time (events around each kernel), same workload ----
    kms = _kernel_pass(ctx, args.steps, lambda: ctx.topk_async(dk, k, olap.DESC, ok, orow, d_rowids=dr))
    peak, peak_kind = _peaks()
    call_ms = float(np.mean(per_launch))
    # the dominant kernel: the streaming filter when the plan has one (it
    # reads every key once), else the select kernel (which then does)
    top = "topk_filter_ms" if "topk_filter_ms" in kms else "topk_select_ms"
    kern_ms = kms[top]
    algo_bytes = n * w
    achieved = algo_bytes / (kern_ms * 1e-3) / 1e9
    traffic = args.traffic
    if traffic is None and top == "topk_filter_ms" and k == 1000 and args.dist == "uniform" \
            and args.filter == "regs" and args.rowids == "explicit":
        traffic = FILTER_DRAM_BYTES_PER_KEY[args.key_type] * n if args.key_type in FILTER_DRAM_BYTES_PER_KEY \
            else None
    line = {
        "metric": METRIC, "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"i64": "int64", "f32": "float32", "f64": "float64", "u64": "uint64",
                                       "i32": "int32", "u32": "uint32"}[args.key_type], "data": "synthetic",
        "config": {"workload": f"topk_{args.key_type}_{args.dist}_n2^{args.log2n}_k{k}_desc", "n": n, "k": k,
                   "order": "desc", "rowids": args.rowids,
                   "l2": f"inputs larger than L2 ({n * w / 2**30:.2f} GiB keys)",
                   "cpu_affinity": affinity,
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": {"topk_filter_ms": "olap::topk_filter_regs_kernel" if args.filter == "regs"
                                else "olap::topk_filter_bulk_kernel",
                                "topk_select_ms": "olap::topk_select_kernel"}[top],
                     "algorithmic_bytes_per_launch": algo_bytes,
                     "bytes_per_unit": f"{w} per key read once", "kernel_ms": kern_ms,
                     "kernel_ms_all": kms, "call_ms": call_ms,
                     "call_ms_median": _median_p95(per_launch)[0], "call_ms_p95": _median_p95(per_launch)[1],
                     "call_frac": algo_bytes / (call_ms * 1e-3) / 1e9 / peak,
                     "timing": "CUDA events around each kernel on the library stream, "
                               f"{args.steps} further steps after the timed region",
                     "filter": args.filter, "last_launch": phases,
                     "geometry": {"tile": args.tile, "stages": args.stages, "ctas_per_sm": args.ctas_per_sm}},
        "e2e": {"value": e2e_value, "unit": "Gkeys/s",
                "h2d_bytes_per_step": n * w + (4 * n if hr is not None and not rid_in_place else 0),
                "rowid_bytes_read_in_place": 4 * int(e2e_info["candidates"]) if rid_in_place else 0,
                "d2h_bytes_per_step": k * (w + 4) + 4, "ms_per_step": e2e_s * 1e3,
                "rowids": ("explicit, in pinned host memory: the keys are copied, the kernels read the "
                           "candidates' row-ids in place" if rid_in_place else
                           "explicit (keys and row-ids cross the link)") if hr is not None else "implicit (keys only)",
                "keys_only": e2e_keys_only},
        # the library's own count over the timed regions of `value` and `e2e`
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if "single" in workloads:
        line["single"] = single_leg(args, ctx, torch)
    if "link" in workloads:
        line["link"] = link_leg(torch)
    if "join" in workloads:
        del dk, hk, dr, hr
        torch.cuda.empty_cache()
        line["join"] = join_leg(args, ctx, torch, world)
    if "pair" in workloads:
        torch.cuda.empty_cache()
        line["pair"] = pair_leg(args, ctx, torch, world)
    if "joincells" in workloads:
        torch.cuda.empty_cache()
        line["join_cells"] = join_cells_leg(args, ctx, torch, world)
    if "topkcells" in workloads:
        torch.cuda.empty_cache()
        line["topk_cells"] = topk_cells_leg(args, ctx, torch, world)
    if "batched" in workloads:
        torch.cuda.empty_cache()
        line["batched"] = batched_leg(args, ctx, torch)
    if "fullrow" in workloads:
        torch.cuda.empty_cache()
        line["fullrow"] = fullrow_leg(args, ctx, torch)
    if "gate" in workloads:
        torch.cuda.empty_cache()
        line["gate"] = gate_leg(args, ctx, torch)
    if "serving" in workloads:
        torch.cuda.empty_cache()
        line["serving"] = serving_leg(args, ctx, torch)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n, k)
        line["cpu_baseline"]["host"] = _host_info()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--k", type=int, default=1000)
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--key-type", default="i64", choices=["i64", "f32", "f64", "u64", "i32", "u32"])
    ap.add_argument("--dist", default="uniform", choices=["uniform", "ascending", "dup1024"])
    ap.add_argument("--rowids", default="explicit", choices=["implicit", "explicit"],
                    help="explicit (the configured workload): uint32 row-ids 0..N-1 passed with the keys (read "
                         "on the device only for survivors; they cross the link in the end-to-end figure)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the timed kernel, if captured")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload",
                    default="topk,single,pair,link,join,joincells,topkcells,batched,fullrow,gate,serving",
                    help="comma list: topk (the headline value), single (2^20-key query latency), link (pinned "
                         "copy bandwidth), join (probe sub-object), batched (executor), "
                         "pair (two-column key Top-K), joincells (every join cell), topkcells (every Top-K "
                         "cell at 2^log2n), fullrow (full-row vs "
                         "key-only transfer), "
                         "gate (break-even validation), "
                         "serving (gated vs always-on stream)")
    ap.add_argument("--join-cell", default="unique,uniform,0.9",
                    help="build multiplicity (unique|mult14), probe distribution (uniform|zipf), hit rate")
    ap.add_argument("--join-log2b", type=int, default=24)
    ap.add_argument("--join-log2p", type=int, default=28)
    ap.add_argument("--join-steps", type=int, default=50)
    ap.add_argument("--join-cell-steps", type=int, default=5, help="timed probes per cell of the joincells leg")
    ap.add_argument("--topk-cell-steps", type=int, default=10, help="timed calls per cell of the topkcells leg")
    ap.add_argument("--join-traffic", type=float, default=None)
    ap.add_argument("--gate-points", type=int, default=16, help="N grid points of the gate leg (1e3..1e8)")
    ap.add_argument("--fullrow-payload", type=int, default=100, help="payload bytes per row of the full-row leg")
    ap.add_argument("--batch-overlap", type=int, default=0, help="0: Top-K then probe kernel; 1: side by side")
    ap.add_argument("--batch-topk-ctas", type=int, default=0, help="batched Top-K CTAs per SM (0 = 2)")
    ap.add_argument("--fullrow-reps", type=int, default=11)
    ap.add_argument("--gate-reps", type=int, default=5)
    ap.add_argument("--join-partitions", type=int, default=0,
                    help="0 automatic, 1 direct probe, 2..256 forced partition count")
    ap.add_argument("--join-loads", type=int, default=0, help="bucket reads: 0 auto, 1 via L1, 2 L2 only")
    ap.add_argument("--l2-fetch", type=int, default=0, help="L2 fetch granularity to set (0 = leave)")
    ap.add_argument("--batch-topk", type=int, default=4096)
    ap.add_argument("--batch-probe", type=int, default=1024)
    ap.add_argument("--batch-reps", type=int, default=10)
    ap.add_argument("--serve-requests", type=int, default=100_000)
    ap.add_argument("--serve-arena", type=int, default=100_000_000)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-pin", type=int, default=0,
                    help="1: the serving host engine computes on its own cores (the last serve-cpu-workers), the "
                         "GPU path's threads on the rest")
    ap.add_argument("--host-threads", type=int, default=12,
                    help="host engine threads of the gate and full-row legs (the engine alone on the host)")
    ap.add_argument("--serve-cpu-workers", type=int, default=4,
                    help="host engine workers (and its threads); the rest of the host's cores stage the GPU "
                         "requests' copies")
    ap.add_argument("--serve-budget-gb", type=int, default=40)
    ap.add_argument("--serve-margin", type=float, default=0.0)
    ap.add_argument("--serve-cal-points", type=int, default=18)
    ap.add_argument("--serve-host", default="staged", choices=["auto", "staged"],
                    help="how the serving contexts copy pageable keys: direct device access where supported, "
                         "or CPU staging through pinned buffers")
    ap.add_argument("--serve-topk-cpu", default="max", choices=["best", "max"],
                    help="Top-K CPU model of the serving gate: the better-fitting form, or both forms' maximum")
    ap.add_argument("--tile", type=int, default=0, help="bulk-copy bytes (0 = library default)")
    ap.add_argument("--stages", type=int, default=0, help="copies in flight per CTA (0 = default)")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="resident CTAs per SM (0 = default)")
    ap.add_argument("--filter", default="regs", choices=["bulk", "regs"],
                    help="Top-K streaming pass: register loads (default) or bulk-copy ring")
    return ap


def main():
    args = build_parser().parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
