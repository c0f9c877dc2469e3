#!/usr/bin/env python
"""Benchmark of the gapped k-mer kernel engine on one node.

One step = the whole hot path over one batch of synthetic datasets: g-mer
packing, every (m, mask) sort and run-length pass, the on-chip C_m
accumulation with inclusion-exclusion and K = sum h_m N_m, mirroring and
fp64 normalisation.  Default workload: five independent DNA datasets
(N = 500, 1000, 2000, 3000, 4000; lengths uniform in [100, 300]; GC 0.4;
g = 10, k = 6, M = 4), all in one batched call replayed from a CUDA graph.

Prints one JSON line.  ``value`` is Gram entries per second (sum of N_i^2
over datasets and ranks / step time) with inputs resident on the device;
``e2e`` is the same metric through the host-buffer C ABI call, host<->device
copies included (outputs written into host arrays the caller keeps across
calls).  ``--impl reference`` times the CPU oracle instead.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W]
                       [--workload dna_large|dna_toy|protein|text]
                       [--impl ours|reference]
Multi-GPU: launch with torch.distributed.run, one rank per GPU; each rank
processes its own independently seeded batch (weak scaling, no collective
on the data path).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1704_07468_gb300 import synth  # noqa: E402

METRIC = "Gram entries/s"
UNIT = "entries/s"
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2
SMEM_BANKS = 32              # shared-memory banks per SM (32-bit each)


def make_workload(name, rank=0, dna_sizes=None, n=None):
    """-> (description, sigma, g, k, list of (codes, offsets)); ``n``
    overrides the sequence count of the single-dataset workloads (smaller
    cases for profiling)."""
    off = 1000 * rank
    if name == "dna_large":
        sizes = tuple(dna_sizes) if dna_sizes else synth.DNA_LARGE_SIZES
        seeds = tuple(s + off for s in (2, 3, 4, 5, 6))[:len(sizes)]
        sets = synth.dna_large(seeds=seeds, sizes=sizes)
        return (f"DNA large-M batched: {len(sizes)} datasets, N={'/'.join(map(str, sizes))}, "
                "lengths U[100,300], GC 0.4, g=10 k=6 (M=4)", 4, 10, 6, sets)
    if name == "dna_toy":
        nn = n or 200
        return (f"DNA toy: N={nn}, length 100, uniform ACGT, g=7 k=5 (M=2)", 4, 7, 5,
                [synth.dna_toy(seed=1 + off, n=nn)])
    if name == "protein":
        nn = n or 3312
        return (f"protein: N={nn}, sigma=20, Dirichlet(2) residues, log-normal lengths "
                "(median 300, clipped [50,1000]), g=8 k=4 (M=4)", 20, 8, 4,
                [synth.protein(seed=7 + off, n=nn)])
    if name == "text":
        nn = n or 6000
        return (f"text: N={nn}, sigma=36, Zipf(1.1) symbols, lengths U[200,2000], "
                "g=8 k=5 (M=3)", 36, 8, 5, [synth.text(seed=8 + off, n=nn)])
    raise SystemExit(f"unknown workload {name}")


def reduce_max(value, device=None):
    """Max of a float over all ranks (one all-reduce, outside timed regions)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], 0, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = max(smax, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def oracle_sample(sigma, g, k, sets, rows_per_set, threads):
    """Time the CPU oracle on a bounded sample: `rows_per_set` rows of the
    largest dataset against all of its columns.  Returns (entries/s,
    seconds, description)."""
    import oracle

    codes, off = max(sets, key=lambda s: len(s[1]))
    n = len(off) - 1
    rows = np.linspace(0, n - 1, rows_per_set).round().astype(np.int32)
    t0 = time.perf_counter()
    oracle.gram(codes, off, g, k, rows=rows, threads=threads)
    dt = time.perf_counter() - t0
    desc = (f"{rows_per_set} evenly spaced rows x all {n} columns of the N={n} dataset, "
            f"plus the {n} self-profiles for the diagonal")
    return rows_per_set * n / dt, dt, desc


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    desc, sigma, g, k, sets = make_workload(args.workload, 0, args.dna_sizes)
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    rows = args.ref_rows
    oracle_sample(sigma, g, k, sets, 2, threads)  # warm-up (page-in)
    vals, secs = [], []
    for _ in range(args.warmup):
        oracle_sample(sigma, g, k, sets, rows, threads)
    for _ in range(args.steps):
        v, dt, sdesc = oracle_sample(sigma, g, k, sets, rows, threads)
        vals.append(v)
        secs.append(dt)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * float(np.mean(secs)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sdesc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# DRAM bytes (read + write) per unit of work from one ncu capture of the
# same kernels on a smaller case (one step of the DNA N = 2000 dataset, see
# profiles/traffic_dna_2000.md), scaled to a launch of the bench by its
# units; traffic grows in proportion to them.
NCU_BYTES_PER_UNIT = {
    "accumulate": ((1.3201e9 + 0.0887e9) / 8.292e8, "pair update"),
    "dense_gemm": ((1.7618e9 + 0.0001e9) / 3.442e12, "flop"),
    "dense_scatter": ((0.0217e9 + 1.6969e9) / 1.762e9, "byte of A"),
    "sort_pass": ((1.1911e9 + 0.9131e9) / 2.493e9, "algorithmic byte"),
    "run_length": ((1.1498e9 + 0.6941e9) / 1.344e9, "algorithmic byte"),
}
NCU_SOURCE = {name: "profiles/traffic_dna_2000.md (scaled by units)" for name in NCU_BYTES_PER_UNIT}


def kernel_rooflines(timings, work, peaks, sm_count, smem_atomic_peak=None):
    """Roofline entry per timed stage with a known algorithmic work figure.

    ``work`` holds the engine's own counts for the step: pair updates of
    the accumulation, algorithmic sort bytes, dense-contraction flops
    (upper triangle, unpadded) and issued flops, dense A bytes."""
    out = {}
    timings = dict(timings)
    if "diag" in timings and "combine" in timings:
        (ms_d, n_d), (ms_c, n_c) = timings.pop("diag"), timings.pop("combine")
        timings["diag+combine"] = (ms_d + ms_c, max(n_d, n_c))
    # The dense contraction runs on e4m3 operands: its peak is the measured
    # bf16 figure times the nominal e4m3 / bf16 ratio (4.5 / 2.25 PFLOP/s).
    tensor_peak = peaks.get("bf16_tflops", 1900.0) * 2.0
    for name, (ms, n) in timings.items():
        sec = ms / 1000.0
        if sec <= 0:
            continue
        e = None
        if name == "accumulate" and work["pairs"] > 0:
            # One 32-bit shared-memory atomic add per pair update; peak =
            # the conflict-free shared-atomic rate measured on this GPU by
            # the library's probe (else banks x SMs x max SM clock).
            if smem_atomic_peak:
                peak, src = smem_atomic_peak / 1e12, "measured: conflict-free shared-memory atomic adds (gakco_measure_smem_atomics)"
            else:
                peak = SMEM_BANKS * sm_count * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
                src = "derived: 32 shared-memory banks x SMs x max SM clock"
            a = work["pairs"] / sec / 1e12
            e = {"bound": "alu", "achieved": a, "peak": peak, "unit": "Tupdates/s",
                 "kernel": "k_accum", "peak_source": src}
        elif name == "sort_pass" and work["sort_bytes"] > 0:
            a = work["sort_bytes"] / sec / 1e9
            e = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "kernel": "k_upsweep + k_digit_scan + k_digit_base + k_downsweep"}
        elif name == "dense_gemm" and work["dense_flops"] > 0:
            a = work["dense_flops"] / sec / 1e12
            e = {"bound": "tensor", "achieved": a, "peak": tensor_peak, "unit": "TFLOP/s",
                 "kernel": "k_dense_gemm",
                 "issued_tflops": work["dense_issued"] / sec / 1e12,
                 "dtype": "e4m3 x e4m3 -> f32",
                 "peak_source": "measured bf16 burst x 2 (nominal e4m3/bf16 ratio)"}
        elif name == "dense_scatter" and work["dense_bytes"] > 0:
            a = work["dense_bytes"] / sec / 1e9
            e = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "kernel": "k_dense_scatter"}
        elif name == "run_length" and work.get("rle_bytes", 0) > 0:
            a = work["rle_bytes"] / sec / 1e9
            e = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "kernel": "k_rle_count + k_rle_scan + k_rle_emit_gram + k_rle_fix"}
        elif name == "pack" and work.get("pack_bytes", 0) > 0:
            a = work["pack_bytes"] / sec / 1e9
            e = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "kernel": "k_pack"}
        elif name == "diag+combine" and work.get("combine_bytes", 0) > 0:
            a = work["combine_bytes"] / sec / 1e9
            e = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "kernel": "k_diag + k_combine"}
        if e is None:
            continue
        e["frac"] = e["achieved"] / e["peak"]
        e["traffic"] = None
        units = {"accumulate": work["pairs"], "dense_gemm": work["dense_flops"],
                 "dense_scatter": work["dense_bytes"], "sort_pass": work["sort_bytes"],
                 "run_length": work.get("rle_bytes", 0)}.get(name)
        if name in NCU_BYTES_PER_UNIT and units:
            per, unit = NCU_BYTES_PER_UNIT[name]
            e["traffic"] = per * units / n          # bytes per launch
            e["traffic_source"] = f"{NCU_SOURCE[name]}: {per:.4g} B per {unit}"
        e["launch_ms"] = ms / n
        e["launches"] = n
        out[name] = e
    return out


def run_configs(pkg, names, steps, flush):
    """The other single-GPU workloads, each in its own batched device call
    (autotuned, replayed from its graph, K and Khat outputs): ms per step,
    CUDA events on the calling stream, the L2 flush between steps."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    out = {}
    for name in names:
        desc, sigma, g, k, sets = make_workload(name)
        ns = [len(o) - 1 for _, o in sets]
        d_codes = [torch.from_numpy(c).to(dev) for c, _ in sets]
        d_K = [torch.empty((n, n), dtype=torch.int32, device=dev) for n in ns]
        d_Kh = [torch.empty((n, n), dtype=torch.float64, device=dev) for n in ns]
        offs = [o for _, o in sets]
        with pkg.gakco_create(sigma, g, k) as ctx:
            ctx.autotune_device([t.data_ptr() for t in d_codes], offs, stream=stream.cuda_stream)

            def step():
                ctx.gram_batch_device([t.data_ptr() for t in d_codes], offs,
                                      [t.data_ptr() for t in d_K], [t.data_ptr() for t in d_Kh],
                                      None, stream=stream.cuda_stream)
            for _ in range(3):
                step()
            ms = []
            for _ in range(steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step()
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            t = float(np.mean(ms))
            out[name] = {"ms_per_step": t, "entries_per_s": sum(n * n for n in ns) / (t / 1000.0),
                         "dense_problems": int(ctx.get_stat("dense_problems")), "workload": desc}
        del d_codes, d_K, d_Kh
        torch.cuda.empty_cache()
    return out


def run_gemm_rate(pkg, peaks):
    """The dense GEMM alone on full tiles: a kernel-only Gram (level 4 of
    DNA g = 10, k = 6, dense: 210 masks x 4096 6-mers = 860160 columns) of
    4096 uniform sequences of length 200 is 136 macro tiles of 256 x 256
    outputs, 6720 K-stages each, one per CTA.  Issued flops over the
    launch's event time give the repo's own tcgen05 e4m3 rate; scaled by
    152 / 136 busy SMs it estimates the device rate."""
    import torch

    codes, off = synth.fixed_length(77, 4096, 200, 4)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream().cuda_stream
    d_codes = torch.from_numpy(codes).to(dev)
    K = torch.empty((4096, 4096), dtype=torch.int32, device=dev)
    with pkg.gakco_create(4, 10, 6) as ctx:
        ctx.set_option("dense", 2)
        ctx.set_option("kernel_only", 1)
        ctx.set_option("profile", 1)
        best = None
        for _ in range(4):
            ctx.gram_device(d_codes.data_ptr(), off, K.data_ptr(), stream=stream)
            torch.cuda.synchronize()
            ms = ctx.kernel_timings()["dense_gemm"][0]
            best = ms if best is None else min(best, ms)
        issued = ctx.get_stat("dense_issued_flops")
        alg = ctx.get_stat("dense_flops")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    rate = issued / (best / 1000.0) / 1e12
    derived = peaks.get("bf16_tflops", 1900.0) * 2.0
    return {"workload": "kernel-only Gram, DNA g=10 k=6, 4096 x length-200 sequences: 136 full macro tiles",
            "gemm_ms": best, "issued_tflops": rate, "algorithmic_tflops": alg / (best / 1000.0) / 1e12,
            "busy_sms": 136, "sms": sms, "device_rate_estimate_tflops": rate * sms / 136,
            "derived_peak_tflops": derived, "estimate_vs_derived": rate * sms / 136 / derived}


def run_serve(pkg, n_requests, warmup):
    """Serving workload: the protein training set resident on the device, a
    Poisson stream of test batches (mean 5 ms apart, 1-256 sequences each),
    replayed in real time.  Continuous batching (submit / poll) against the
    plain per-request path (each request alone, synchronously, in arrival
    order).  Latency = completion - scheduled arrival."""
    tr = synth.protein()
    reqs = synth.serve_requests(warmup + n_requests, seed=9)
    ntr = len(tr[1]) - 1

    def summarize(lat, rows, span):
        lat = np.sort(np.asarray(lat))
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "rows_per_s": rows / span,
                "gram_entries_per_s": rows * ntr / span}

    ctx = pkg.gakco_create(20, 8, 4)
    ctx.fit(*tr)
    # Warm the slots and the synchronous path.
    for _, c, o in reqs[:3]:
        ctx.cross_fitted(c, o)
    t0 = time.perf_counter()
    i, pending, lat, lib_lat, rows = 0, {}, [], [], 0
    first = last = None
    while i < len(reqs) or pending:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i][0] <= now:
            pending[ctx.submit(reqs[i][1], reqs[i][2])] = (i, reqs[i][0])
            i += 1
        for t in list(pending):
            out = ctx.poll(t, 0)
            if out is None:
                continue
            idx, arr = pending.pop(t)
            done = time.perf_counter() - t0
            if idx >= warmup:
                lat.append((done - arr) * 1e3)
                lib_lat.append(out["latency_ms"])
                rows += len(reqs[idx][2]) - 1
                first = arr if first is None else min(first, arr)
                last = done if last is None else max(last, done)
        time.sleep(0.0001)
    cb = summarize(lat, rows, last - first)
    cb["submit_to_done_p50_ms"] = float(np.percentile(lib_lat, 50))
    cb["batches"] = int(ctx.get_stat("served_batches"))
    # Plain per-request path on the same arrivals.
    t0 = time.perf_counter()
    lat, rows, first, last = [], 0, None, None
    for idx, (arr, c, o) in enumerate(reqs):
        now = time.perf_counter() - t0
        if now < arr:
            time.sleep(arr - now)
        ctx.cross_fitted(c, o)
        done = time.perf_counter() - t0
        if idx >= warmup:
            lat.append((done - arr) * 1e3)
            rows += len(o) - 1
            first = arr if first is None else min(first, arr)
            last = done
    plain = summarize(lat, rows, last - first)
    # Saturated load: every request queued at once (throughput ceiling).
    sat_reqs = reqs[warmup:]
    sat_rows = sum(len(o) - 1 for _, _, o in sat_reqs)
    t0 = time.perf_counter()
    tickets = [ctx.submit(c, o) for _, c, o in sat_reqs]
    for t in tickets:
        ctx.poll(t, -1)
    sat_cb = sat_rows / (time.perf_counter() - t0)
    t0 = time.perf_counter()
    for _, c, o in sat_reqs:
        ctx.cross_fitted(c, o)
    sat_plain = sat_rows / (time.perf_counter() - t0)
    ctx.close()
    return {"saturated_rows_per_s": {"continuous_batching": sat_cb, "plain_per_request": sat_plain},
            "workload": f"protein train N={ntr} resident; {n_requests} requests after {warmup} warm-up, "
                        "Poisson mean 5 ms, 1-256 sequences each, normalised K(test, train) rows",
            "continuous_batching": cb, "plain_per_request": plain}


def run_extend(pkg, sigma, g, k, sets, add=100):
    """Adding `add` sequences (the tail of the largest dataset) to a fitted
    set of the rest, against a fresh Gram computation on the union."""
    codes, off = max(sets, key=lambda s: len(s[1]))
    n = len(off) - 1
    cut = n - add
    old = (codes[:off[cut]], off[:cut + 1])
    new = (codes[off[cut]:], off[cut:] - off[cut])
    with pkg.gakco_create(sigma, g, k) as ctx:
        ctx.set_option("dense", 1)
        ctx.gram(codes, off, khat=True)           # warm the full-size plan
        t0 = time.perf_counter()
        full = ctx.gram(codes, off, khat=True)
        t_full = time.perf_counter() - t0
        ctx.fit(*old)
        ctx.extend(*new)                           # warm-up (refits on the union)
        ctx.fit(*old)
        t0 = time.perf_counter()
        rows = ctx.extend(*new)
        t_ext = time.perf_counter() - t0
    return {"workload": f"add {add} sequences to a fitted set of {cut} (DNA large-M N={n} dataset)",
            "extend_ms": 1000 * t_ext, "fresh_gram_ms": 1000 * t_full,
            "equal_to_fresh_rows": bool(np.array_equal(rows["K"], full["K"][cut:]) and
                                        np.array_equal(rows["Khat"], full["Khat"][cut:])),
            "timing": "wall clock through the host-buffer C ABI, copies and the merge of the new sequences into the index included"}


def run_nsweep(pkg):
    """Kernel time as N grows at fixed length l = 100 (Section 3.2, Fig. 5(c)):
    DNA with an unknown-base symbol (sigma = 5), protein, text."""
    out = []
    for name, sigma, g, k in (("dna_sigma5", 5, 10, 6), ("protein", 20, 8, 4), ("text", 36, 8, 5)):
        for n in (100, 250, 500, 750):
            codes, off = synth.fixed_length(1000 + n, n, 100, sigma)
            with pkg.gakco_create(sigma, g, k) as ctx:
                ctx.set_option("dense", 1)
                ctx.gram(codes, off)
                ts = []
                for _ in range(3):
                    t0 = time.perf_counter()
                    ctx.gram(codes, off)
                    ts.append(time.perf_counter() - t0)
            out.append({"data": name, "N": n, "l": 100, "g": g, "k": k, "ms": 1000 * min(ts)})
    return out


def run_ours(args):
    import torch

    import paper_1704_07468_gb300 as pkg
    from paper_1704_07468_gb300 import build as lib_build

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    lib_build.build()
    desc, sigma, g, k, sets = make_workload(args.workload, rank, args.dna_sizes, args.n)
    ns = [len(o) - 1 for _, o in sets]
    entries = float(sum(n * n for n in ns))

    ctx = pkg.gakco_create(sigma, g, k)
    n_masks = sum(1 for m in range(g - k + 1) for _ in range(__import__("math").comb(g, m)))
    d_codes = [torch.from_numpy(c).to(dev) for c, _ in sets]
    d_K = [torch.empty((n, n), dtype=torch.int32, device=dev) for n in ns]
    d_Kh = [torch.empty((n, n), dtype=torch.float64, device=dev) for n in ns]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    offs = [o for _, o in sets]

    def step():
        ctx.gram_batch_device([t.data_ptr() for t in d_codes], offs,
                              [t.data_ptr() for t in d_K], [t.data_ptr() for t in d_Kh],
                              None, stream=stream.cuda_stream)

    tuned = "defaults"
    if not args.no_autotune:
        t_tune = time.perf_counter()
        tuned = ctx.autotune_device([t.data_ptr() for t in d_codes], offs,
                                    stream=stream.cuda_stream)
        tuned += f" ({time.perf_counter() - t_tune:.1f} s, before warm-up)"
    if args.dense is not None:
        ctx.set_option("dense", args.dense)
        tuned += f"; dense={args.dense} set by --dense"
    if args.sort is not None:
        ctx.set_option("sort", args.sort)
        tuned += f"; sort={args.sort} set by --sort"
    for kv in args.set or []:
        name, val = kv.split("=", 1)
        ctx.set_option(name, int(val))
        tuned += f"; {name}={val} set by --set"

    for _ in range(max(args.warmup, 3)):
        step()
    launches = int(ctx.get_stat("launches"))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        times.append((a, b))
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in times]
    step_ms = float(np.mean(ms))
    replay = int(ctx.get_stat("graph_replay"))
    pairs = ctx.get_stat("pair_updates")
    work = {"pairs": pairs, "sort_bytes": ctx.get_stat("sort_bytes"),
            "dense_flops": ctx.get_stat("dense_flops"),
            "dense_issued": ctx.get_stat("dense_issued_flops"),
            "dense_bytes": ctx.get_stat("dense_bytes"),
            "rle_bytes": ctx.get_stat("rle_bytes"),
            "pack_bytes": ctx.get_stat("pack_bytes"),
            "combine_bytes": ctx.get_stat("combine_bytes"),
            "dense_problems": int(ctx.get_stat("dense_problems"))}
    if ws > 1:
        step_ms = reduce_max(step_ms, dev)
        torch.distributed.barrier()
    value = entries * ws / (step_ms / 1000.0)

    # Per-kernel timing: one profiled replay of the same step (every launch
    # bracketed by CUDA events on the engine's stream).
    ctx.set_option("profile", 1)
    step()
    torch.cuda.synchronize()
    timings = ctx.kernel_timings()
    ctx.set_option("profile", 0)
    step()  # re-capture the graph for the calls below

    # End to end through the host-buffer C ABI (copies included).
    # Two untimed calls first: the first plans and captures the host-buffer
    # call's graph, the second still met a slow outlier at times.
    # The outputs go into host arrays the caller keeps across calls (every
    # call still copies all of K and Khat back).
    e2e_out = [{"K": np.empty((n, n), np.int32), "Khat": np.empty((n, n), np.float64)} for n in ns]
    e2e_ms = []
    for i in range(max(1, args.e2e_steps) + 2):
        t0 = time.perf_counter()
        ctx.gram_batch(sets, khat=True, nm=False, out=e2e_out)
        dt = (time.perf_counter() - t0) * 1000.0
        if i > 1:
            e2e_ms.append(dt)
    # Median: a single host-side stall (seen at times on the shared box, tens
    # of ms) would otherwise dominate the mean; every call is listed in calls_ms.
    e2e_step = float(np.median(e2e_ms))
    h2d = int(sum(c.nbytes + o.nbytes for c, o in sets))
    d2h = int(sum(n * n * (4 + 8) for n in ns))

    # Plain per-mask GPU path (same kernels, one mask per launch, global
    # atomics, no graph) for the batched-vs-plain comparison.
    plain = None
    if args.plain_steps > 0:
        pctx = pkg.gakco_create(sigma, g, k)
        pctx.set_option("engine", 1)
        pk = [torch.empty((n, n), dtype=torch.int32, device=dev) for n in ns]
        pkh = [torch.empty((n, n), dtype=torch.float64, device=dev) for n in ns]

        def pstep():
            pctx.gram_batch_device([t.data_ptr() for t in d_codes], offs,
                                   [t.data_ptr() for t in pk], [t.data_ptr() for t in pkh],
                                   None, stream=stream.cuda_stream)
        pstep()
        pms = []
        for _ in range(args.plain_steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pstep()
            b.record(stream)
            torch.cuda.synchronize()
            pms.append(a.elapsed_time(b))
        same = all(torch.equal(x, y) for x, y in zip(pk, d_K))
        plain = {"value": entries / (float(np.mean(pms)) / 1000.0), "unit": UNIT,
                 "ms_per_step": float(np.mean(pms)),
                 "mask_passes_per_s": len(sets) * n_masks / (float(np.mean(pms)) / 1000.0),
                 "launches": int(pctx.get_stat("launches")),
                 "bit_identical_K": bool(same)}
        pctx.close()

    # Kernel-only mode (K = C_M: the level-M masks alone), same options,
    # reported beside the full path; the headline value is the full path.
    konly = None
    if args.kernel_only_steps > 0:
        kctx = pkg.gakco_create(sigma, g, k)
        if not args.no_autotune:
            kctx.autotune_device([t.data_ptr() for t in d_codes], offs, stream=stream.cuda_stream)
        if args.dense is not None:
            kctx.set_option("dense", args.dense)
        if args.sort is not None:
            kctx.set_option("sort", args.sort)
        for kv in args.set or []:
            name, val = kv.split("=", 1)
            kctx.set_option(name, int(val))
        kctx.set_option("kernel_only", 1)
        kk = [torch.empty((n, n), dtype=torch.int32, device=dev) for n in ns]
        kkh = [torch.empty((n, n), dtype=torch.float64, device=dev) for n in ns]

        def kstep():
            kctx.gram_batch_device([t.data_ptr() for t in d_codes], offs,
                                   [t.data_ptr() for t in kk], [t.data_ptr() for t in kkh],
                                   None, stream=stream.cuda_stream)
        for _ in range(3):
            kstep()
        kms = []
        for _ in range(args.kernel_only_steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            kstep()
            b.record(stream)
            torch.cuda.synchronize()
            kms.append(a.elapsed_time(b))
        kmean = float(np.mean(kms))
        konly = {"value": entries * ws / (kmean / 1000.0), "unit": UNIT, "ms_per_step": kmean,
                 "mask_passes_per_step": int(kctx.get_stat("mask_passes")),
                 "bit_identical_K": bool(all(torch.equal(x, y) for x, y in zip(kk, d_K))),
                 "what": "K = C_M (Eq. 6 coefficients = Eq. 8 level-M coefficients): level-M masks only"}
        kctx.close()

    # Roofline of every stage with a work figure; the dominant one is the
    # headline entry.
    peaks, peak_kind = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    try:
        smem_peak = pkg.gakco_measure_smem_atomics(stream.cuda_stream)
        smem_random = pkg.gakco_measure_smem_atomics(stream.cuda_stream, random_columns=True)
    except pkg.GakcoError:
        smem_peak = smem_random = None
    roofs = kernel_rooflines(timings, work, peaks, sm_count, smem_peak)
    if smem_random and "accumulate" in roofs:
        # Context: the same adds at random columns (the accumulation's pattern).
        roofs["accumulate"]["random_column_rate"] = smem_random / 1e12
        roofs["accumulate"]["frac_of_random_column_rate"] = roofs["accumulate"]["achieved"] / (smem_random / 1e12)
    total_ms = sum(v[0] for v in timings.values())
    for name, e in roofs.items():
        e["peak_kind"] = peak_kind
        e["share_of_step"] = e["launch_ms"] * e["launches"] / total_ms
    dom_name = max(timings.items(), key=lambda kv: kv[1][0])[0]
    if dom_name in roofs:
        roof = dict(roofs[dom_name])
    else:
        roof = {"bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": None, "traffic": None, "kernel": dom_name, "peak_kind": peak_kind,
                "share_of_step": timings[dom_name][0] / total_ms}
    roof["stage"] = dom_name
    # Every stage in one compact table (ms, share of the serialised step,
    # fraction of its roofline), kept inside the roofline entry.
    roof["stages"] = {}
    for name, (t_ms, _) in sorted(timings.items(), key=lambda kv: -kv[1][0]):
        r = roofs.get(name) or roofs.get("diag+combine" if name in ("diag", "combine") else "")
        row = {"ms": round(t_ms, 3), "share": round(t_ms / total_ms, 3)}
        if r is not None:
            row.update({"frac": round(r["frac"], 3), "bound": r["bound"],
                        "achieved": round(r["achieved"], 3), "unit": r["unit"]})
        roof["stages"][name] = row

    configs = None
    if args.config_steps > 0 and rank == 0 and args.workload == "dna_large":
        configs = run_configs(pkg, ("dna_toy", "protein", "text"), args.config_steps, flush)

    serve = None
    if args.serve_requests > 0 and rank == 0:
        serve = run_serve(pkg, args.serve_requests, args.serve_warmup)
    extend = run_extend(pkg, sigma, g, k, sets) if args.extras and rank == 0 else None
    gemm_rate = run_gemm_rate(pkg, peaks) if args.extras and rank == 0 else None
    if gemm_rate and "dense_gemm" in roofs:
        # Context: the same kernel's issued rate on full tiles (all SMs busy,
        # scaled from the busy ones), beside the derived e4m3 peak.
        rate = gemm_rate["device_rate_estimate_tflops"]
        roofs["dense_gemm"]["measured_kernel_rate_tflops"] = rate
        roofs["dense_gemm"]["frac_of_measured_kernel_rate"] = roofs["dense_gemm"]["achieved"] / rate
        if roof.get("stage") == "dense_gemm":
            roof.update({k: roofs["dense_gemm"][k] for k in ("measured_kernel_rate_tflops",
                                                              "frac_of_measured_kernel_rate")})
    nsweep = run_nsweep(pkg) if args.extras and rank == 0 else None

    cpu = None
    if rank == 0 and ws == 1 and args.cpu_rows > 0:
        import oracle
        oracle.build()
        thr = oracle.default_threads()
        v, dt, sdesc = oracle_sample(sigma, g, k, sets, args.cpu_rows, thr)
        cpu = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sdesc,
               "seconds": dt}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": desc, "datasets": ns, "g": g, "k": k, "sigma": sigma,
                   "outputs": "K int32 + Khat fp64 per dataset",
                   "l2": "256 MiB write between timed steps",
                   "graph_replay": bool(replay), "parallelism": f"replicas x{ws} (weak)",
                   "autotune": tuned, "dense_problems": work["dense_problems"]},
        "mask_passes_per_s": len(sets) * n_masks * ws / (step_ms / 1000.0),
        "pair_updates_per_step": pairs,
        "plain_gpu": plain,
        "kernel_only": konly,
        "serve": serve,
        "extend": extend,
        "nsweep_l100": nsweep,
        "e2e": {"value": entries * ws / (e2e_step / 1000.0), "unit": UNIT,
                "ms_per_step": e2e_step, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "calls_ms": [round(v, 3) for v in e2e_ms]},
        "gpu_launches": launches * args.steps,
        "kernel_ms": {kname: {"ms": v[0], "launches": v[1]} for kname, v in timings.items()},
        "roofline": roof,
        "roofline_stages": roofs,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "configs": configs,
        "gemm_rate": gemm_rate,
    }
    # Compact figures last on the line, so that they survive a reader that
    # keeps only the end of it.
    summ = {"ms_per_step": round(step_ms, 3), "e2e_ms": round(e2e_step, 3),
            "mask_passes_per_s": round(line["mask_passes_per_s"], 1)}
    if plain:
        summ.update({"plain_per_mask_ms": round(plain["ms_per_step"], 2),
                     "batched_vs_plain": round(plain["ms_per_step"] / step_ms, 2),
                     "plain_mask_passes_per_s": round(plain["mask_passes_per_s"], 1),
                     "plain_bit_identical": plain["bit_identical_K"]})
    if konly:
        summ["kernel_only_ms"] = round(konly["ms_per_step"], 3)
    if serve:
        cb, pl = serve["continuous_batching"], serve["plain_per_request"]
        summ["serve"] = {"p50_ms": round(cb["p50_ms"], 2), "p99_ms": round(cb["p99_ms"], 2),
                         "rows_per_s": round(cb["rows_per_s"]),
                         "plain_p50_ms": round(pl["p50_ms"], 2), "plain_p99_ms": round(pl["p99_ms"], 2),
                         "plain_rows_per_s": round(pl["rows_per_s"]),
                         "saturated_rows_per_s": round(serve["saturated_rows_per_s"]["continuous_batching"]),
                         "plain_saturated_rows_per_s": round(serve["saturated_rows_per_s"]["plain_per_request"])}
    if configs:
        summ["configs_ms"] = {n: round(v["ms_per_step"], 3) for n, v in configs.items()}
    if gemm_rate:
        summ["gemm_issued_tflops_full_tiles"] = round(gemm_rate["issued_tflops"], 1)
    summ["frac"] = {n: r["frac"] for n, r in roof["stages"].items() if "frac" in r}
    line["summary"] = summ
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="dna_large")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-rows", type=int, default=64)
    ap.add_argument("--ref-rows", type=int, default=16)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--extras", type=int, default=1,
                    help="1: also time adding sequences and the N-sweep at l = 100")
    ap.add_argument("--kernel-only-steps", type=int, default=3,
                    help="also time the K = C_M mode (level-M masks only); 0 to skip")
    ap.add_argument("--dense", type=int, default=None, choices=[0, 1, 2],
                    help="dense-level mode after autotuning: 0 never, 1 cost model, 2 every qualifying level")
    ap.add_argument("--config-steps", type=int, default=5,
                    help="also time the toy, protein and text workloads (dna_large run only); 0 to skip")
    ap.add_argument("--sort", type=int, default=None, choices=[0, 1],
                    help="sort after autotuning: 0 upsweep/scan/downsweep per pass, 1 onesweep")
    ap.add_argument("--set", action="append", metavar="NAME=VALUE",
                    help="engine option (paper_1704_07468_gb300.OPT name) set after autotuning; repeatable")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--n", type=int, default=None,
                    help="sequences of the dna_toy / protein / text workload (smaller cases for profiling)")
    ap.add_argument("--dna-sizes", type=lambda v: [int(t) for t in v.split(",")], default=None,
                    help="subset of DNA dataset sizes (small cases for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
