#!/usr/bin/env python3
"""Benchmark of the fused sufficient-statistics pass on the paper's Table 1 workload.

Workload: Table 1 (arxiv 2604.23826), n = 1e9 rows per GPU, seed 1, generated on
the device into the L32 columnar layout (60 B/row; A int64, nine int32 columns,
cotC and J float64).  One step = the whole hot path over the table: the exact
fused pass (n, s = X^T 1, S = X^T X; bit-exact for the integer-valued columns)
followed by finalize (mean, covariance, correlation, PCA eigenpairs) and the
device-to-host read of its result.  Inputs (60 GB) are larger than L2, so no
flush is needed between steps.

  python bench.py [--gpus N --steps K --warmup W]        the CUDA path (default N=1)
  python bench.py --impl reference                       the CPU oracle as the reference arm

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
import math

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rows/s and HBM GB/s (% of roofline) for fused sums+XᵀX at stated accuracy vs plain FP64"
UNIT = "rows/s"
SEED = 1
BYTES_PER_ROW = {0: 60, 1: 44}

# DRAM traffic per row of the exact pass (dram__bytes_read.sum + dram__bytes_write.sum over
# the rows of one ncu capture, profiles/exact_pass_table1_L32_n5e7.md), with the hash of the
# kernel sources it was taken on; reported as null once those sources change.
NCU_TRAFFIC = {"bytes_per_row": 60.069, "src_hash": "1f417e2a986ce63b", "layout": "L32"}


# DRAM traffic of the FP32 split passes (BF16x3) from one ncu capture each on a smaller case:
# reads per algorithmic byte (they grow with the rows) plus the per-launch slot writes (fixed);
# profiles/wide2_pairs_p256_bf16x3_n4e6.md and profiles/narrow_tcgen05_p64_bf16x3_n8e6.md.
NCU_TRAFFIC_SPLIT = {
    "wide2": {"read_per_byte": 4220192000 / 4096000000, "write_bytes": 126807296,
              "files": ("k_wide2.cu", "tc05.cuh", "common.cuh"), "src_hash": "6c2a6506838f0ead"},
    "narrow": {"read_per_byte": 2074298000 / 2048000000, "write_bytes": 31283200,
               "files": ("k_narrow.cu", "tc05.cuh", "common.cuh"), "src_hash": "22da905282b4366e"},
}


def split_traffic(kind: str, algorithmic_bytes: int):
    """Traffic of one split-pass launch scaled from its capture, or None if the sources changed."""
    t = NCU_TRAFFIC_SPLIT[kind]
    h = hashlib.sha256()
    for f in t["files"]:
        with open(os.path.join(ROOT, "paper_2604_23826_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != t["src_hash"]:
        return None
    return t["read_per_byte"] * algorithmic_bytes + t["write_bytes"]


def kernel_src_hash() -> str:
    h = hashlib.sha256()
    for f in ("k_exact.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2604_23826_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=float, default=1e9, help="rows per GPU")
    ap.add_argument("--layout", choices=("L32", "L16"), default="L32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-detail", action="store_true",
                    help="cpu_baseline also times the oracle with one thread and the histogram oracle at n = 1e10")
    ap.add_argument("--no-comparator", action="store_true")
    ap.add_argument("--chunk-rows", type=int, default=1 << 24)
    ap.add_argument("--exact-shape", type=int, default=-1,
                    help="launch shape of the exact pass (-1: the library default; 0-3: stats.h)")
    ap.add_argument("--workload", choices=("table1", "tables4096", "wide256", "f32table", "table1_1e10", "table1_file",
                                                "table1_csv"),
                    default="table1",
                    help="table1: the headline line; tables4096 / wide256 / f32table: the FP32 workloads")
    ap.add_argument("--p", type=int, default=64, help="f32table: columns")
    ap.add_argument("--ntables", type=int, default=4096)
    ap.add_argument("--wave-gb", type=float, default=64.0)
    ap.add_argument("--mode", default=None, help="tables4096 / wide256: BF16X3, BF16X4, FP32, FP64S; tables4096 also FP64")
    ap.add_argument("--tune", choices=("off", "cached", "measure"), default="off",
                    help="tables4096: batched-launch tuning (off: library defaults; cached: a cached choice for "
                         "this device and library build, measured first if there is none; measure: re-measure on "
                         "the first wave)")
    ap.add_argument("--by-width", action="store_true",
                    help="tables4096: also time each width class's tables alone (reported, not the headline)")
    ap.add_argument("--oracle-check", choices=("none", "quick", "full"), default="quick",
                    help="tables4096: tables compared with the CPU oracle (quick: 64 of <= 1e6 rows and 16 "
                         "larger, stratified by rows; full: every table of <= 1e6 rows and 64 larger); "
                         "wide256: rows of the prefix compared (quick 1e6, full 1e7)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


def bind_host_to_gpu(local_rank: int) -> dict:
    """Restrict this process to the host cores attached to its GPU (sysfs local_cpulist of the
    GPU's PCI function, intersected with the cores the process may use), so that pinned host
    buffers allocated afterwards are placed on the GPU's own CPU socket: a host -> device copy
    from the other socket crosses the CPU-to-CPU link first.  Returns what was done."""
    info = {"bound": False}
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader",
                              "-i", gpu_index(local_rank)], capture_output=True, text=True, timeout=20)
        bus = out.stdout.strip().splitlines()[0].strip().lower()
        dom, rest = bus.split(":", 1)
        sysdir = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}"
        info["pci"] = bus
        with open(os.path.join(sysdir, "local_cpulist")) as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        allowed = os.sched_getaffinity(0)
        info["_previous"] = allowed
        both = cpus & allowed
        info["local_cpus"] = spec
        if both and both != allowed:
            os.sched_setaffinity(0, both)
            info["bound"] = True
        info["cores"] = len(both or allowed)
    except Exception as e:  # no nvidia-smi or sysfs entry: leave the affinity alone
        info["error"] = type(e).__name__
    return info


def h2d_copy_rate(torch, host, chunk_rows: int, dev, reps: int = 5) -> float:
    """Host-to-device rate of the e2e path's own copies without the pass: the same pinned host
    columns, one cudaMemcpyAsync per column per chunk of chunk_rows rows into two alternating
    device staging buffers, on a side stream (as stats_accumulate_host issues them); GB/s,
    best of `reps` passes over the whole table."""
    n = host[0].numel()
    stage = [[torch.empty(min(chunk_rows, n), dtype=h.dtype, device=dev) for h in host] for _ in range(2)]
    s = torch.cuda.Stream(device=dev)
    best = float("inf")
    with torch.cuda.stream(s):
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            b = 0
            for r0 in range(0, n, chunk_rows):
                rows = min(chunk_rows, n - r0)
                for h, d in zip(host, stage[b]):
                    d[:rows].copy_(h[r0:r0 + rows], non_blocking=True)
                b ^= 1
            e1.record(s)
            s.synchronize()
            best = min(best, e0.elapsed_time(e1))
    nbytes = sum(h.numel() * h.element_size() for h in host)
    del stage
    return nbytes / (best / 1e3) / 1e9


def read_only_peak_gbs(torch, dev, gib: int = 8) -> float:
    """A read-only streaming rate of this GPU's HBM for the roofline's side figure: torch's sum
    over a `gib` GiB float32 buffer (inputs far larger than L2), best of 5, CUDA events."""
    x = torch.empty((gib << 30) // 4, dtype=torch.float32, device=dev)
    best = float("inf")
    for _ in range(6):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        x.sum()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del x
    torch.cuda.empty_cache()
    return (gib << 30) / (best / 1e3) / 1e9


def gemm_tflops(torch, dev, dtype, n: int) -> float:
    """Dense GEMM rate of this GPU in `dtype` (torch.matmul, n^3, best of 3, CUDA events): the
    measured FP64 rate that the plain FP64 comparator is set against."""
    a = torch.randn((n, n), dtype=dtype, device=dev)
    b = torch.randn((n, n), dtype=dtype, device=dev)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ----------------------------------------------------------------------------- CPU oracle runs
def oracle_sample(seconds: float, row0: int = 0):
    """Time the per-row oracle (exact sums + exact centering + Jacobi) on a sample of
    Table 1 sized for about `seconds` of CPU work; returns (rows, seconds, threads)."""
    import oracle as O
    threads = O.default_threads()
    t0 = time.perf_counter()
    O.stats_table1(SEED, 200_000, row0=row0, threads=threads)
    dt = max(time.perf_counter() - t0, 1e-3)
    n = int(min(max(200_000 * seconds / dt, 200_000), 2e9))
    t0 = time.perf_counter()
    st = O.stats_table1(SEED, n, row0=row0, threads=threads)
    _, cov, _ = O.analysis_from_stats(st)
    O.jacobi(cov)
    return n, time.perf_counter() - t0, threads


def oracle_detail(threads: int) -> dict:
    """The oracle's rates on the host cores: the per-row oracle at n = 1e6 with all threads and
    with one, and the exact histogram oracle (a count-only pass over the 6000 (B, C, D) cells)
    on the n = 1e10 table with all threads, its closed forms checked."""
    import oracle as O
    out = {}
    for th in (threads, 1):
        t0 = time.perf_counter()
        O.stats_table1(SEED, 1_000_000, threads=th)
        dt = time.perf_counter() - t0
        out[f"per_row_n1e6_threads{th}"] = {"rows_per_s": 1e6 / dt, "s": dt}
    n10 = 10**10
    t0 = time.perf_counter()
    st = O.stats_table1_hist(2, n10, threads=threads)
    dt = time.perf_counter() - t0
    out["histogram_n1e10"] = {"rows_per_s": n10 / dt, "s": dt, "threads": threads,
                              "closed_forms": bool(st.n == n10 and st.s[0] == n10 * (n10 + 1) // 2 and
                                                   st.S[0][0] == n10 * (n10 + 1) * (2 * n10 + 1) // 6)}
    return out


def run_reference(args, rank: int):
    if rank != 0:
        return
    import oracle as O
    threads = O.default_threads()
    # size each step for ~8 s of CPU work
    t0 = time.perf_counter()
    O.stats_table1(SEED, 200_000, threads=threads)
    dt = max(time.perf_counter() - t0, 1e-3)
    n_step = int(min(max(200_000 * 8.0 / dt, 200_000), 1e9))
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        st = O.stats_table1(SEED, n_step, row0=i * n_step, threads=threads)
        _, cov, _ = O.analysis_from_stats(st)
        O.jacobi(cov)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    value = n_step / (ms / 1000.0)
    sample = (f"Table 1 rows, seed {SEED}, {n_step} rows per step (a bounded sample of the {int(args.n)}-row "
              f"workload): per-row exact sums (__int128 / double-double), exact centering, Jacobi")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int128/f64x2", "data": "synthetic",
           "config": {"workload": f"table1_n{int(args.n)}_seed{SEED}_{args.layout}", "rows_per_step": n_step,
                      "p": 12, "where": "host CPU cores"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- the CUDA path
def run_ours(args, rank: int, world: int, local_rank: int):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_23826_gb300 as G

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    layout = G.STATS_T1_L32 if args.layout == "L32" else G.STATS_T1_L16
    n = int(args.n)
    bpr = BYTES_PER_ROW[layout]
    row0 = rank * n  # weak scaling: each rank its own contiguous block of the global table
    stream = torch.cuda.current_stream()

    # ---- generation (a1), untimed in the metric, reported separately ----
    cols = G.alloc_table1(n, layout)
    G.stats_gen_table1(SEED, row0, min(n, 1 << 20), layout, cols)  # warm the generator
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record()
    G.stats_gen_table1(SEED, row0, n, layout, cols)
    g1.record()
    torch.cuda.synchronize()
    gen_ms = g0.elapsed_time(g1)

    cfg = G.stats_table1_config(layout, world * n, G.STATS_EXACT)
    ctx = G.stats_init(cfg)
    G.stats_set_exact_shape(ctx, args.exact_shape)
    pass_events = []
    from paper_2604_23826_gb300 import shard
    combined = {}

    def step(record: bool):
        G.stats_reset(ctx)
        if record:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        G.stats_accumulate(ctx, cols, n, stream)
        if record:
            e1.record(stream)
            pass_events.append((e0, e1))
        if world == 1:
            return G.stats_finalize(ctx, 0)
        # the one exchange of the sharded pass: every rank's (n, s, S) exported, gathered in rank
        # order, imported and merged; the analysis is of the whole table
        merged = shard.combine_contexts(ctx)
        try:
            an = G.stats_finalize(merged, 0)
            combined["raw"] = G.stats_raw(merged)
            return an
        finally:
            merged.close()

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(gpu_index(local_rank))
    sampler.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    elapsed_ms = t0.elapsed_time(t1)
    kernel_ms = sum(a.elapsed_time(b) for a, b in pass_events) / len(pass_events)

    # correctness of what was timed: identifier closed forms of this rank's rows and, with
    # several ranks, of the whole table's rows in the combined statistics
    raw = G.stats_raw(ctx)
    lo, hi = row0, row0 + n
    checks = {"sumA": raw.s_exact[0] == hi * (hi + 1) // 2 - lo * (lo + 1) // 2,
              "sumA2": raw.S_exact[0][0] == (hi * (hi + 1) * (2 * hi + 1) - lo * (lo + 1) * (2 * lo + 1)) // 6,
              "n": raw.n == n}
    if world > 1:
        g, N = combined["raw"], world * n
        checks["combined_n"] = g.n == N
        checks["combined_sumA"] = g.s_exact[0] == N * (N + 1) // 2
        checks["combined_sumA2"] = g.S_exact[0][0] == N * (N + 1) * (2 * N + 1) // 6

    # ---- the plain FP64 comparator on the same table (the metric's "vs plain FP64") ----
    comparator = None
    if not args.no_comparator:
        with G.stats_init(G.stats_table1_config(layout, row0 + n, G.STATS_FP64)) as c64:
            G.stats_accumulate(c64, cols, n, stream)
            G.stats_sync(c64)
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            G.stats_reset(c64)
            f0.record(stream)
            G.stats_accumulate(c64, cols, n, stream)
            f1.record(stream)
            G.stats_sync(c64)
            fp64_ms = f0.elapsed_time(f1)
            r64 = G.stats_raw(c64)
        import math
        relA = abs(r64.S[0, 0] - float(raw.S_exact[0][0])) / float(raw.S_exact[0][0])
        comparator = {"kernel": "plain FP64 CUDA cores (raw moments)", "rows_per_s": n / (fp64_ms / 1e3),
                      "ms": fp64_ms, "speedup_exact_vs_fp64": fp64_ms / kernel_ms,
                      "fp64_rel_err_sumA2": relA if math.isfinite(relA) else None}
        # its own roofline: 90 multiply-adds per row (12 sums + 78 products) against the FP64
        # rate measured here (cuBLAS DGEMM, 4096^3, best of 3)
        try:
            fp64_peak = gemm_tflops(torch, dev, torch.float64, 4096)
            achieved = 180.0 * n / (fp64_ms / 1e3) / 1e12
            comparator.update({"fp64_tflops_achieved": achieved, "fp64_tflops_peak_measured": fp64_peak,
                               "fp64_frac": achieved / fp64_peak})
        except RuntimeError:
            pass

    # ---- e2e: the same step through host (pinned) buffers, copies inside the timed region ----
    e2e = None
    if not args.no_e2e:
        n_e2e = n
        host = None
        affinity = bind_host_to_gpu(local_rank)
        while host is None and n_e2e >= (1 << 24):
            try:
                host = [torch.empty(n_e2e, dtype=c.dtype, pin_memory=True) for c in cols]
            except RuntimeError:
                host = None
                n_e2e //= 2
        if host is not None:
            for h, c in zip(host, cols):
                h.copy_(c[:n_e2e])
            torch.cuda.synchronize()

            def step_e2e():
                G.stats_reset(ctx)
                G.stats_accumulate_host(ctx, host, n_e2e, args.chunk_rows, stream)
                return G.stats_finalize(ctx, 0)

            step_e2e()
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            k_e2e = max(3, min(args.steps, 10))
            h0 = torch.cuda.Event(enable_timing=True)
            h1 = torch.cuda.Event(enable_timing=True)
            h0.record(stream)
            for _ in range(k_e2e):
                step_e2e()
            h1.record(stream)
            torch.cuda.synchronize()
            e2e_ms = h0.elapsed_time(h1) / k_e2e
            # the e2e path's roofline: its own copies (same buffers, chunks and copy calls) alone
            h2d_gbs = h2d_copy_rate(torch, host, args.chunk_rows, dev)
            pa = 11
            T = 12 * 13 // 2
            result_bytes = 8 * (1 + 12 + T + 2 * 12 + 2 * T + pa + 3 * pa * pa + pa + 8) + 8 + 4
            e2e = {"value": n_e2e / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": n_e2e * bpr,
                   "d2h_bytes_per_step": result_bytes, "rows": n_e2e, "ms_per_step": e2e_ms, "steps": k_e2e,
                   "h2d_GBps_achieved": n_e2e * bpr / (e2e_ms / 1e3) / 1e9, "h2d_GBps_measured_copy": h2d_gbs,
                   "h2d_copy_probe": "the same pinned columns copied chunk by chunk (one cudaMemcpyAsync per "
                                     "column per chunk, two staging buffers) with no pass, best of 5",
                   "h2d_frac": (n_e2e * bpr / (e2e_ms / 1e3) / 1e9) / h2d_gbs,
                   "api": "stats_accumulate_host (pinned host columns, double-buffered chunks) + stats_finalize",
                   "host_affinity": {k: v for k, v in affinity.items() if not k.startswith("_")}}
            del host
        else:
            e2e = {"value": None, "unit": UNIT, "note": "pinned host allocation failed"}
        if affinity.get("_previous"):
            os.sched_setaffinity(0, affinity["_previous"])  # the CPU baseline gets every core again

    # ---- reduce over ranks ----
    t = torch.tensor([elapsed_ms, kernel_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ok = torch.tensor([1 if all(checks.values()) else 0], device=dev)
        dist.all_reduce(ok, op=dist.ReduceOp.MIN)
        checks["all_ranks"] = bool(ok.item())
        if e2e and e2e.get("value"):
            ev = torch.tensor([n_e2e / e2e["value"]], dtype=torch.float64, device=dev)
            dist.all_reduce(ev, op=dist.ReduceOp.MAX)
            e2e["value"] = world * n_e2e / ev.item()
    elapsed_ms, kernel_ms = t.tolist()
    ms_per_step = elapsed_ms / args.steps

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows, secs, threads = oracle_sample(15.0)
        cpu = {"value": rows / secs, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{rows} Table 1 rows (seed {SEED}) of the {n}-row workload: per-row exact "
                         f"__int128/double-double sums, exact centering, Jacobi; {secs:.1f} s"}
        if args.oracle_detail:
            cpu["detail"] = oracle_detail(threads)

    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    if not peak:
        peak = 6800.0
    achieved = n * bpr / (kernel_ms / 1e3) / 1e9
    read_peak = None
    try:
        read_peak = read_only_peak_gbs(torch, dev)
    except RuntimeError:  # no room for the 8 GiB buffer next to the table
        pass
    traffic = None
    if (NCU_TRAFFIC["bytes_per_row"] and NCU_TRAFFIC["src_hash"] == kernel_src_hash()
            and NCU_TRAFFIC["layout"] == args.layout and args.exact_shape in (-1, 0)):
        traffic = NCU_TRAFFIC["bytes_per_row"] * n
    out = {
        "metric": METRIC, "value": world * n / (ms_per_step / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"table1_n{n:.0e}_seed{SEED}_{args.layout}".replace("+", ""), "rows_per_gpu": n,
                   "p": 12, "layout": args.layout, "bytes_per_row": bpr, "mode": "STATS_EXACT",
                   "exact_shape": args.exact_shape,
                   "step": "exact fused pass + finalize (mean, cov, corr, PCA) + D2H of the result",
                   "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"rows sharded over {world} rank(s)" + (
                       "; each step ends with the export / rank-ordered gather / import + merge of the ranks' "
                       "statistics, then the analysis of the whole table" if world > 1 else "")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_src, "traffic": traffic,
                     "kernel": ("exact_tc_kernel<ConvT1> (tcgen05)" if args.exact_shape == 3 else
                                "exact_pass_kernel<ConvT1>"), "kernel_ms": kernel_ms,
                     "algorithmic_bytes": n * bpr,
                     "peak_nominal": 8000.0, "frac_nominal": achieved / 8000.0,
                     "peak_read_only_measured": read_peak,
                     "frac_read_only": achieved / read_peak if read_peak else None},
        "e2e": e2e,
        "cpu_baseline": cpu,
        # per step: the pass and finalize, plus one merge launch per other rank's image
        "gpu_launches": (2 + (world - 1)) * args.steps,
        "clocks": clocks,
        "generator": {"rows_per_s": n / (gen_ms / 1e3), "GB_per_s_written": n * bpr / (gen_ms / 1e3) / 1e9},
        "comparator": comparator,
        "checks": checks,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()

# ----------------------------------------------------------------------------- FP32 workloads
MODE_NAMES = {"BF16X3": "STATS_BF16X3", "BF16X4": "STATS_BF16X4", "FP32": "STATS_FP32", "FP64S": "STATS_FP64_SHIFTED",
              "FP64": "STATS_FP64"}
MODE_KERNEL = {"BF16X3": "split_kernel (mma.sync bf16)", "BF16X4": "split_kernel (mma.sync bf16)",
               "FP32": "core_kernel<float>", "FP64S": "core_kernel<double> (shifted; fp64 kernel for p <= 12)",
               "FP64": "core_kernel<double> (raw moments, the paper's plain FP64 kernel; fp64 kernel for p <= 12)"}


def _base_line(args, world, metric, value, ms_per_step, config, roofline, clocks, launches, extra):
    out = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config, "roofline": roofline,
           "e2e": None, "cpu_baseline": None, "gpu_launches": launches, "clocks": clocks}
    out.update(extra)
    return out


def run_tables(args, rank: int, world: int, local_rank: int):
    """Many independent FP32 tables (shapes of the batched workload), one batched call per wave."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_23826_gb300 as G
    from paper_2604_23826_gb300 import inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    seed = 3
    mode_name = args.mode or "BF16X4"
    mode = getattr(G, MODE_NAMES[mode_name])
    params = inputs.many_tables_shapes(seed, args.ntables)
    mine = list(range(rank, len(params), world))  # weak scaling: tables dealt round-robin to ranks
    groups = inputs.waves([params[t] for t in mine], int(args.wave_gb * 1e9))
    groups = [[mine[i] for i in g] for g in groups]
    ctxs = {t: G.stats_init(G.Config([G.STATS_F32] * params[t][1], mode, [0] * params[t][1])) for t in mine}
    rows_total = sum(params[t][0] for t in mine)
    bytes_total = sum(4 * params[t][0] * params[t][1] for t in mine)
    # each table is a [p, ld] block with ld = n rounded up to 4 floats: 16-byte aligned columns
    ld = {t: (params[t][0] + 3) // 4 * 4 for t in mine}
    buf = torch.empty(max(sum(params[t][1] * ld[t] for t in g) for g in groups), dtype=torch.float32, device=dev)

    def materialise(g):
        views, off = [], 0
        for t in g:
            n, p, mu, sd = params[t]
            blk = buf[off:off + p * ld[t]].view(p, ld[t])
            inputs.gen_table(torch, n, p, mu, sd, 1_000_003 * seed + t, dev, out=blk[:, :n])
            views.append(blk[:, :n])
            off += p * ld[t]
        return views

    tuning = None
    if args.tune != "off":
        from paper_2604_23826_gb300 import tune
        g0 = groups[0]
        views = materialise(g0)
        tuning = tune.autotune_batched([ctxs[t] for t in g0], [[x[j] for j in range(x.shape[0])] for x in views],
                                       [params[t][0] for t in g0], stream=stream, workload=f"tables{args.ntables}",
                                       force=args.tune == "measure")
        for t in g0:
            G.stats_reset(ctxs[t])
    wave_ms = []
    host_ms = []
    # per wave: one pivot launch + one batched launch per tile width present (32: p <= 32, 64: p = 64);
    # the CUDA-core modes run one pass per table (shifted: after its pivot launch)
    launches_per_step = (sum(1 + len({32 if params[t][1] <= 32 else 64 for t in g}) for g in groups)
                         if mode_name.startswith("BF16") else len(mine) * (1 if mode_name == "FP64" else 2))

    def step(record: bool):
        for t in mine:
            G.stats_reset(ctxs[t])
        total = 0.0
        for g in groups:
            views = materialise(g)
            # column pointers (integers) built before the timed region
            cols = [[x.data_ptr() + 4 * x.stride(0) * j for j in range(x.shape[0])] for x in views]
            tabs = [ctxs[t] for t in g]
            rows = [params[t][0] for t in g]
            batch = G.BatchArgs(tabs, cols, rows)  # argument arrays, like the pointers, built outside
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h0 = time.perf_counter()
            G.stats_accumulate_batched(batch, stream=stream)
            if record:
                host_ms.append((time.perf_counter() - h0) * 1e3)
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        if record:
            wave_ms.append(total)

    for _ in range(args.warmup):
        step(False)
    sampler = ClockSampler(gpu_index(local_rank))
    sampler.start()
    time.sleep(0.3)
    for _ in range(args.steps):
        step(True)
    clocks = sampler.stop()
    ms = sum(wave_ms) / len(wave_ms)
    by_width = None
    if args.by_width:
        # each width class's tables alone, wave by wave (the batched call then runs that class's
        # launches only): where the step's time goes
        by_width = {}
        for w in (8, 16, 32, 64):
            w_ms, w_bytes = 0.0, 0
            for g in groups:
                sel = [i for i, t in enumerate(g) if (8 if params[t][1] <= 8 else 16 if params[t][1] <= 16 else
                                                      32 if params[t][1] <= 32 else 64) == w]
                if not sel:
                    continue
                views = materialise(g)
                tabs = [g[i] for i in sel]
                for t in tabs:
                    G.stats_reset(ctxs[t])
                cols = [[views[i].data_ptr() + 4 * views[i].stride(0) * j for j in range(views[i].shape[0])]
                        for i in sel]
                batch = G.BatchArgs([ctxs[t] for t in tabs], cols, [params[t][0] for t in tabs])
                best = float("inf")
                for _ in range(3):
                    for t in tabs:
                        G.stats_reset(ctxs[t])
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    G.stats_accumulate_batched(batch, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                w_ms += best
                w_bytes += sum(4 * params[t][0] * params[t][1] for t in tabs)
            pk = measured_peaks().get("hbm_gbs") or 6800.0
            by_width[w] = {"ms": w_ms, "bytes": w_bytes, "GB_per_s": w_bytes / (w_ms / 1e3) / 1e9,
                           "frac": w_bytes / (w_ms / 1e3) / 1e9 / pk, "share_of_step": w_ms / ms}
        # the contexts hold partial rows now: one more full step restores every table's statistics
        step(False)
    # finalize of every table (reported, outside the pass time): one batched call
    f0 = time.perf_counter()
    finals = G.stats_finalize_batched([ctxs[t] for t in mine])
    fin_ms = (time.perf_counter() - f0) * 1e3
    worst_mean_rel = 0.0
    for t, an in zip(mine, finals):
        n, p, mu, sd = params[t]
        mu32, sd32 = np.float32(mu).astype(np.float64), np.float32(sd).astype(np.float64)
        worst_mean_rel = max(worst_mean_rel, float(np.max(np.abs(an.mean - mu32) / sd32)) * math.sqrt(n))
    oracle_check = None
    tables_cpu = None
    if args.oracle_check != "none" and rank == 0:
        # the same tables regenerated (same seeds, same values), copied back, and the oracle's
        # two-pass covariance compared with the batched pass's result
        import oracle as O
        spec = {"quick": dict(n_small=64, n_large=16), "full": dict(n_small=None, n_large=64)}[args.oracle_check]
        pick = set(inputs.check_sample([params[t] for t in mine], **spec))
        pick = {mine[i] for i in pick}
        fin_of = dict(zip(mine, finals))
        worst, worst_t, o_secs = 0.0, None, 0.0
        for g in groups:
            if not pick.intersection(g):
                continue
            views = materialise(g)
            for t, v in zip(g, views):
                if t not in pick:
                    continue
                H = v.cpu().numpy()
                o0 = time.perf_counter()
                cov = O.cov_twopass_columns([H[j].astype(np.float64) for j in range(H.shape[0])])
                o_secs += time.perf_counter() - o0
                err = float(np.linalg.norm(fin_of[t].cov - cov) / np.linalg.norm(cov))
                if err >= worst:
                    worst, worst_t = err, t
        tables_cpu = {"value": int(sum(params[t][0] for t in pick)) / max(o_secs, 1e-9), "unit": "rows/s",
                      "cores": O.default_threads(), "kind": "oracle",
                      "sample": f"the oracle's two-pass covariance (double-double) of {len(pick)} of the tables "
                                f"({args.oracle_check} sample), {o_secs:.1f} s"}
        oracle_check = {"cov_rel_vs_oracle": worst, "tables": len(pick),
                        "rows": int(sum(params[t][0] for t in pick)),
                        "worst_table": {"index": worst_t, "n": params[worst_t][0], "p": params[worst_t][1]},
                        "sample": args.oracle_check + ": " + ("64 tables of <= 1e6 rows and 16 larger, stratified"
                                                             " by rows" if args.oracle_check == "quick" else
                                                             "every table of <= 1e6 rows and 64 larger, "
                                                             "stratified by rows"),
                        "oracle_s": o_secs, "tolerance": 2e-6}
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") or 6800.0
    achieved = bytes_total / (ms / 1e3) / 1e9
    t_ms = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    ms_all = t_ms.item()
    rows_all = sum(params[t][0] for t in range(len(params)))
    config = {"workload": f"tables{args.ntables}_seed{seed}_f32_{mode_name}", "tables": args.ntables,
              "rows_total": rows_all, "bytes_total": sum(4 * n * p for n, p, _, _ in params),
              "n_range": [1e3, 1e7], "p_choices": [8, 16, 32, 64], "mode": MODE_NAMES[mode_name],
              "waves": len(groups), "wave_gb_max": args.wave_gb,
              "step": "batched fused pass over every table (one launch per wave and tile size); "
                      "inputs regenerated per wave outside the timed region",
              "l2": "inputs larger than L2 (no flush)", "parallelism": f"tables dealt to {world} rank(s)"}
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback", "traffic": None,
            "kernel": "narrow_kernel (tcgen05; 33-64 columns, 53 % of the bytes) + gram32_kernel (mma.sync; 1-32 "
                      "columns)" if mode_name.startswith("BF16") else MODE_KERNEL[mode_name],
            "kernel_ms": ms, "algorithmic_bytes": bytes_total}
    extra = {"finalize_ms_all_tables_batched": fin_ms,
             "host_ms_per_call": sum(host_ms) / max(1, len(host_ms)),
             "check_means_within_sqrt_n_sigma_units": worst_mean_rel,
             "oracle_check": oracle_check, "tuning": tuning, "by_width": by_width}
    out = _base_line(args, world, "rows/s and HBM GB/s (% of roofline) for fused sums+XᵀX, batched FP32 tables",
                     rows_all / (ms_all / 1e3), ms_all, config, roof, clocks,
                     launches_per_step * args.steps, extra)
    out["cpu_baseline"] = tables_cpu if world == 1 else None
    if rank == 0:
        print(json.dumps(out), flush=True)
    for c in ctxs.values():
        c.close()


def run_wide(args, rank: int, world: int, local_rank: int):
    """One wide correlated FP32 table (n x 256), timed in each FP32 mode."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_23826_gb300 as G
    from paper_2604_23826_gb300 import inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    seed, p = 4, 256
    n = int(args.n) if args.n != 1e9 else 100_000_000
    L, mu = inputs.wide_factor(seed, p)
    X = inputs.gen_wide(torch, n, L, mu, seed * 1_000_003 + rank, dev)
    torch.cuda.synchronize()
    cols = [X[j] for j in range(p)]
    modes = [args.mode] if args.mode else ["BF16X3", "BF16X4", "FP32", "FP64S"]
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") or 6800.0
    tflops = peaks.get("bf16_tflops")
    results = {}
    sampler = ClockSampler(gpu_index(local_rank))
    sampler.start()
    time.sleep(0.3)
    for mname in modes:
        mode = getattr(G, MODE_NAMES[mname])
        nm = n
        steps = args.steps if mname != "FP64S" else 1  # the FP64 pass is FP64-FMA bound: one timed pass
        cm = [c[:nm] for c in cols]
        with G.stats_init(G.Config([G.STATS_F32] * p, mode, [0] * p)) as ctx:
            if mname != "FP64S":
                G.stats_accumulate(ctx, cm, nm, stream)
                G.stats_sync(ctx)
            ev = []
            for _ in range(steps):
                G.stats_reset(ctx)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                G.stats_accumulate(ctx, cm, nm, stream)
                e1.record(stream)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
            # the analysis (mean, cov, corr, PCA) of the accumulated statistics, then a streaming
            # snapshot after 1 % more rows, its eigen-solve seeded by the first one's eigenvectors
            t0 = time.perf_counter()
            an = G.stats_finalize_warm(ctx, 0)
            fin_ms = (time.perf_counter() - t0) * 1e3
            G.stats_accumulate(ctx, [c[:nm // 100] for c in cm], nm // 100, stream)
            G.stats_sync(ctx)
            t0 = time.perf_counter()
            an2 = G.stats_finalize_warm(ctx, 0, an.evecs)
            snap_ms = (time.perf_counter() - t0) * 1e3
        top = np.asarray(an.evals[:10])
        results[mname] = {"rows": nm, "ms": ms, "rows_per_s": nm / (ms / 1e3),
                          "GB_per_s": 4 * p * nm / (ms / 1e3) / 1e9,
                          "hbm_frac": 4 * p * nm / (ms / 1e3) / 1e9 / peak,
                          "top10_eval_rel_to_1_over_k": float(np.max(np.abs(top - 1.0 / np.arange(1, 11)) *
                                                                     np.arange(1, 11))),
                          "finalize_ms": fin_ms, "finalize_sweeps": an.sweeps,
                          "snapshot_seeded_ms": snap_ms, "snapshot_seeded_sweeps": an2.sweeps,
                          "cov": an.cov}
    clocks = sampler.stop()
    if args.oracle_check != "none" and rank == 0:
        # the oracle on a prefix of the same table, against each mode's pass over that prefix
        import oracle as O
        m = min(n, 1_000_000 if args.oracle_check == "quick" else 10_000_000)
        H = X[:, :m].cpu().numpy()
        o0 = time.perf_counter()
        cov_o = O.cov_twopass_columns([H[j].astype(np.float64) for j in range(p)])
        o_secs = time.perf_counter() - o0
        del H
        ev_o = np.linalg.eigvalsh(cov_o)[::-1][:10]
        for mname in modes:
            with G.stats_init(G.Config([G.STATS_F32] * p, getattr(G, MODE_NAMES[mname]), [0] * p)) as ctx:
                G.stats_accumulate(ctx, [c[:m] for c in cols], m, stream)
                an_m = G.stats_finalize(ctx, 0)
            results[mname]["oracle_check"] = {
                "rows": m, "cov_rel_vs_oracle": float(np.linalg.norm(an_m.cov - cov_o) / np.linalg.norm(cov_o)),
                "top10_eval_rel_vs_oracle": float(np.max(np.abs(an_m.evals[:10] - ev_o) / ev_o)),
                "oracle_s": o_secs, "sample": f"the table's first {m} rows on both sides"}
    wide_cpu = None
    if args.oracle_check != "none" and rank == 0 and world == 1:
        wide_cpu = {"value": m / o_secs, "unit": "rows/s", "cores": O.default_threads(), "kind": "oracle",
                    "sample": f"the oracle's two-pass covariance (double-double) of the table's first {m} rows, "
                              f"{o_secs:.1f} s"}
    ref = results.get("FP64S")
    main_mode = modes[0]
    for mname, r in results.items():
        if ref is not None and mname != "FP64S" and r["rows"] == n and ref["rows"] == n:
            r["cov_rel_vs_fp64s"] = float(np.linalg.norm(r["cov"] - ref["cov"]) / np.linalg.norm(ref["cov"]))
    for r in results.values():
        del r["cov"]
    m = results[main_mode]
    flops_row = {"BF16X3": 3, "BF16X4": 4}.get(main_mode, 1) * 2 * (p * (p + 1) // 2 + p)
    config = {"workload": f"wide_n{n:.0e}_p{p}_seed{seed}_f32".replace("+", ""), "rows_per_gpu": n, "p": p,
              "bytes_per_row": 4 * p, "mode": MODE_NAMES[main_mode], "modes_timed": modes,
              "step": "one fused pass over the table", "l2": "inputs larger than L2 (no flush)",
              "parallelism": f"rows sharded, {world} replica(s)"}
    roof = {"bound": "hbm", "achieved": m["GB_per_s"], "peak": peak, "unit": "GB/s", "frac": m["hbm_frac"],
            "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
            "traffic": split_traffic("wide2", 4 * p * n) if main_mode == "BF16X3" and 128 < p <= 256 else None,
            "kernel": (("wide2_kernel (tcgen05 cta_group::2, pairs of SMs, TMEM accumulators)" if 128 < p <= 256 else
                        "wide_kernel (tcgen05, TMEM accumulators)") if main_mode.startswith("BF16") else
                       MODE_KERNEL[main_mode]), "kernel_ms": m["ms"], "algorithmic_bytes": 4 * p * n,
            "tensor_tflops_useful": flops_row * n / (m["ms"] / 1e3) / 1e12, "tensor_peak_tflops": tflops}
    t_ms = torch.tensor([m["ms"]], dtype=torch.float64, device=dev)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    out = _base_line(args, world, "rows/s and HBM GB/s (% of roofline) for fused sums+XᵀX, wide FP32 table",
                     world * n / (t_ms.item() / 1e3), t_ms.item(), config, roof, clocks,
                     (3 if main_mode.startswith("BF16") else 2) * (args.steps if main_mode != "FP64S" else 1),
                     {"modes": results})
    out["cpu_baseline"] = wide_cpu
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_f32table(args, rank: int, world: int, local_rank: int):
    """One FP32 table of the many-tables distribution (independent N(mu_j, sigma_j^2) columns), p columns,
    n rows, stored as a [p, ld] block (ld = n rounded up to 4 floats), timed in one mode."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_23826_gb300 as G
    from paper_2604_23826_gb300 import inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    seed, p = 3, args.p
    n = int(args.n) if args.n != 1e9 else int(16e9 / (4 * p))
    mode_name = args.mode or "BF16X4"
    rng = np.random.default_rng(seed)
    mu, sd = rng.uniform(1e3, 1e5, p), rng.uniform(0.1, 10.0, p)
    ld = (n + 3) // 4 * 4
    blk = torch.empty((p, ld), dtype=torch.float32, device=dev)
    X = inputs.gen_table(torch, n, p, mu, sd, seed * 1_000_003 + rank, dev, out=blk[:, :n])
    cols = [X[j] for j in range(p)]
    with G.stats_init(G.Config([G.STATS_F32] * p, getattr(G, MODE_NAMES[mode_name]), [0] * p)) as ctx:
        for _ in range(args.warmup):
            G.stats_reset(ctx)
            G.stats_accumulate(ctx, cols, n, stream)
        G.stats_sync(ctx)
        sampler = ClockSampler(gpu_index(local_rank))
        sampler.start()
        time.sleep(0.3)
        ev = []
        for _ in range(args.steps):
            G.stats_reset(ctx)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            G.stats_accumulate(ctx, cols, n, stream)
            e1.record(stream)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        clocks = sampler.stop()
        an = G.stats_finalize(ctx)
    ms = sum(a.elapsed_time(b) for a, b in ev) / len(ev)
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") or 6800.0
    gbs = 4 * p * n / (ms / 1e3) / 1e9
    mu32, sd32 = np.float32(mu).astype(np.float64), np.float32(sd).astype(np.float64)
    config = {"workload": f"f32table_p{p}_n{n}_seed{seed}", "rows_per_gpu": n, "p": p, "bytes_per_row": 4 * p,
              "mode": MODE_NAMES[mode_name], "layout": "[p, ld] block, ld = n rounded up to 4",
              "step": "one fused pass over the table", "l2": "inputs larger than L2 (no flush)",
              "parallelism": f"rows sharded, {world} replica(s)"}
    roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
            "traffic": (split_traffic("narrow", 4 * p * n) if mode_name == "BF16X3" and 32 < p <= 64 and n >= (1 << 20)
                        else None),
            "kernel": (("narrow_kernel (tcgen05, 33-64 columns)" if p > 32 and n >= (1 << 20) else
                        "gram32_kernel (register-fragment mma.sync bf16)") if p <= 64 and mode_name.startswith("BF16")
                       else MODE_KERNEL[mode_name]), "kernel_ms": ms, "algorithmic_bytes": 4 * p * n}
    extra = {"check_means_within_sqrt_n_sigma_units": float(np.max(np.abs(an.mean - mu32) / sd32)) * math.sqrt(n)}
    out = _base_line(args, world, "rows/s and HBM GB/s (% of roofline) for fused sums+XᵀX, one FP32 table",
                     world * n / (ms / 1e3), ms, config, roof, clocks,
                     (3 if p <= 64 and mode_name.startswith("BF16") else 2) * args.steps, extra)
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_table1_stream(args, rank: int, world: int, local_rank: int):
    """Table 1 at n = 1e10 rows (seed 2) into ONE context, in 2^28-row device chunks: each chunk
    generated on the device (untimed), then the exact pass over it (timed with CUDA events);
    checked against the closed forms of the identifier column."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_23826_gb300 as G

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    seed = 2
    layout = G.STATS_T1_L32 if args.layout == "L32" else G.STATS_T1_L16
    bpr = BYTES_PER_ROW[layout]
    n = int(args.n) if args.n != 1e9 else 10_000_000_000
    chunk = 1 << 28
    row0 = rank * n
    cols = G.alloc_table1(chunk, layout)
    cfg = G.stats_table1_config(layout, row0 + n, G.STATS_EXACT)
    pass_ms = []
    with G.stats_init(cfg) as ctx:
        for step in range(args.warmup + args.steps):
            G.stats_reset(ctx)
            total = 0.0
            for r in range(0, n, chunk):
                m = min(chunk, n - r)
                G.stats_gen_table1(seed, row0 + r, m, layout, cols)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                G.stats_accumulate(ctx, [c[:m] for c in cols], m, stream)
                e1.record(stream)
                torch.cuda.synchronize()
                total += e0.elapsed_time(e1)
            if step >= args.warmup:
                pass_ms.append(total)
        raw = G.stats_raw(ctx)
        an = G.stats_finalize(ctx, 1)
    ms = sum(pass_ms) / len(pass_ms)
    lo, hi = row0, row0 + n
    checks = {"sumA": raw.s_exact[0] == hi * (hi + 1) // 2 - lo * (lo + 1) // 2,
              "sumA2": raw.S_exact[0][0] == (hi * (hi + 1) * (2 * hi + 1) - lo * (lo + 1) * (2 * lo + 1)) // 6,
              "n": raw.n == n, "corr_diag_one": bool(np.allclose(np.diag(an.corr), 1.0))}
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") or 6800.0
    gbs = n * bpr / (ms / 1e3) / 1e9
    config = {"workload": f"table1_n{n:.0e}_seed{seed}_{args.layout}_chunked".replace("+", ""), "rows_per_gpu": n,
              "p": 12, "layout": args.layout, "bytes_per_row": bpr, "mode": "STATS_EXACT",
              "chunk_rows": chunk, "step": "exact pass over every chunk into one context (generation untimed)",
              "l2": "inputs larger than L2 (no flush)", "parallelism": f"rows sharded, {world} replica(s)"}
    roof = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
            "traffic": (NCU_TRAFFIC["bytes_per_row"] * n if NCU_TRAFFIC["src_hash"] == kernel_src_hash() and
                        NCU_TRAFFIC["layout"] == args.layout else None),
            "kernel": "exact_pass_kernel<ConvT1>", "kernel_ms": ms, "algorithmic_bytes": n * bpr}
    out = _base_line(args, world, METRIC, world * n / (ms / 1e3), ms, config, roof,
                     {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled (long chunked run)"]},
                     ((n + chunk - 1) // chunk) * args.steps, {"checks": checks, "dtype": "int64"})
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_table1_file(args, rank: int, world: int, local_rank: int):
    """Table 1 from a columnar binary file: written once from the generator (untimed), checked
    the paper's way (header, size, layout; rows from the beginning, middle and end against the
    generator), then streamed through pinned chunks into the exact pass (timed, file pages
    cached by the first read)."""
    import tempfile

    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_23826_gb300 as G

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    seed = 1
    layout = G.STATS_T1_L32 if args.layout == "L32" else G.STATS_T1_L16
    bpr = BYTES_PER_ROW[layout]
    n = int(args.n) if args.n != 1e9 else 100_000_000
    row0 = rank * n
    affinity = bind_host_to_gpu(local_rank)
    tmp = tempfile.mkdtemp(prefix="sscol_")
    path = os.path.join(tmp, f"table1_{rank}.sscol")
    try:
        t0 = time.time()
        G.stats_file_write_table1(path, seed, n, layout, row0=row0)
        write_s = time.time() - t0
        t0 = time.time()
        G.stats_file_check_table1(path, seed, layout, rows_per_region=1 << 16, row0=row0)
        check_s = time.time() - t0
        cfg = G.stats_table1_config(layout, row0 + n, G.STATS_EXACT)
        ms = []
        with G.stats_init(cfg) as ctx:
            for step in range(args.warmup + args.steps):
                G.stats_reset(ctx)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                G.stats_accumulate_file(ctx, path, chunk_rows=args.chunk_rows, stream=stream)
                an = G.stats_finalize(ctx, 0)
                e1.record(stream)
                torch.cuda.synchronize()
                if step >= args.warmup:
                    ms.append(e0.elapsed_time(e1))
            raw = G.stats_raw(ctx)
    finally:
        if os.path.exists(path):
            os.remove(path)
        os.rmdir(tmp)
    step_ms = sum(ms) / len(ms)
    lo, hi = row0, row0 + n
    checks = {"sumA": raw.s_exact[0] == hi * (hi + 1) // 2 - lo * (lo + 1) // 2,
              "sumA2": raw.S_exact[0][0] == (hi * (hi + 1) * (2 * hi + 1) - lo * (lo + 1) * (2 * lo + 1)) // 6,
              "n": raw.n == n, "corr_diag_one": bool(np.allclose(np.diag(an.corr), 1.0))}
    gbs = n * bpr / (step_ms / 1e3) / 1e9
    config = {"workload": f"table1_file_n{n:.0e}_seed{seed}_{args.layout}".replace("+", ""), "rows_per_gpu": n,
              "p": 12, "layout": args.layout, "bytes_per_row": bpr, "mode": "STATS_EXACT",
              "chunk_rows": args.chunk_rows,
              "step": "stats_accumulate_file (pread into pinned chunks, H2D, exact pass) + finalize",
              "file": "columnar table file on the box's local disk, pages cached after the write",
              "parallelism": f"rows sharded, {world} replica(s)"}
    out = _base_line(args, world, METRIC, world * n / (step_ms / 1e3), step_ms, config,
                     {"bound": "host file read", "achieved": gbs, "peak": None, "unit": "GB/s", "frac": None,
                      "traffic": None, "kernel": "exact_pass_kernel<ConvT1>", "algorithmic_bytes": n * bpr},
                     {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled (file pass)"]},
                     args.steps * ((n + args.chunk_rows - 1) // args.chunk_rows + 1), {"checks": checks, "dtype": "int64",
                            "file": {"write_s": write_s, "check_s": check_s, "read_GBps": gbs,
                                     "host_affinity": {k: v for k, v in affinity.items() if not k.startswith("_")}}})
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_table1_csv(args, rank: int, world: int, local_rank: int):
    """Table 1 as CSV text, the paper's starting representation: written once from the generator
    (untimed); then (a) the text already in device memory parsed on the GPU into the twelve
    columns, against the exact binary pass over the same rows, and (b) the file streamed into
    the exact pass (pread into pinned chunks, H2D, GPU parse, pass; pages cached by the write)."""
    import tempfile

    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2604_23826_gb300 as G

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    seed = 1
    layout = G.STATS_T1_L32 if args.layout == "L32" else G.STATS_T1_L16
    bpr = BYTES_PER_ROW[layout]
    n = int(args.n) if args.n != 1e9 else 50_000_000
    row0 = rank * n
    bind_host_to_gpu(local_rank)
    tmp = tempfile.mkdtemp(prefix="sscsv_")
    path = os.path.join(tmp, f"table1_{rank}.csv")
    cfg = G.stats_table1_config(layout, row0 + n, G.STATS_EXACT)
    tdt = {G.STATS_I16: torch.int16, G.STATS_I32: torch.int32, G.STATS_I64: torch.int64, G.STATS_F64: torch.float64}

    def timed(fn, reps):
        out = []
        for i in range(args.warmup + reps):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if i >= args.warmup:
                out.append(e0.elapsed_time(e1))
        return sum(out) / len(out), r

    try:
        t0 = time.time()
        G.stats_csv_write_table1(path, seed, n, layout, row0=row0)
        write_s = time.time() - t0
        text_bytes = os.path.getsize(path)
        # (a) device-resident text: a prefix of whole lines of at most 4 GB
        with open(path, "rb") as f:
            f.readline()
            blob = f.read(min(text_bytes, 4 << 30))
        blob = blob[:blob.rfind(b"\n") + 1]
        m = blob.count(b"\n")
        d_text = torch.frombuffer(bytearray(blob), dtype=torch.uint8).to("cuda")
        del blob
        cols = [torch.empty(m, dtype=tdt[d], device="cuda") for d in cfg.dtypes]
        parse_ms, got = timed(lambda: G.stats_csv_parse(d_text, d_text.numel(), cfg.dtypes, cols, m, stream), args.steps)
        assert got == m
        with G.stats_init(cfg) as ctx:
            def bin_pass():
                G.stats_reset(ctx)
                G.stats_accumulate(ctx, cols, m, stream)
            bin_ms, _ = timed(bin_pass, args.steps)
            raw_dev = G.stats_raw(ctx)
        del d_text, cols
        torch.cuda.empty_cache()
        # (b) the file streamed into the exact pass
        with G.stats_init(cfg) as ctx:
            def file_pass():
                G.stats_reset(ctx)
                r = G.stats_accumulate_csv(ctx, path, skip_lines=1, stream=stream)
                G.stats_sync(ctx)
                return r
            file_ms, got = timed(file_pass, args.steps)
            raw = G.stats_raw(ctx)
    finally:
        if os.path.exists(path):
            os.remove(path)
        os.rmdir(tmp)
    lo, hi = row0, row0 + n
    checks = {"rows": got == n, "sumA": raw.s_exact[0] == hi * (hi + 1) // 2 - lo * (lo + 1) // 2,
              "sumA2": raw.S_exact[0][0] == (hi * (hi + 1) * (2 * hi + 1) - lo * (lo + 1) * (2 * lo + 1)) // 6,
              "prefix_sumA": raw_dev.s_exact[0] == (lo + m) * (lo + m + 1) // 2 - lo * (lo + 1) // 2}
    text_per_row = text_bytes / n
    config = {"workload": f"table1_csv_n{n:.0e}_seed{seed}_{args.layout}".replace("+", ""), "rows_per_gpu": n,
              "p": 12, "layout": args.layout, "mode": "STATS_EXACT", "csv_bytes": text_bytes,
              "csv_bytes_per_row": text_per_row, "binary_bytes_per_row": bpr,
              "step": "stats_accumulate_csv (pread into pinned 64 MB chunks, H2D, GPU parse, exact pass) + sync",
              "file": "CSV on the box's local disk, pages cached after the write",
              "parallelism": f"rows sharded, {world} replica(s)"}
    extra = {"checks": checks, "write_s": write_s,
             "device_parse": {"rows": m, "ms": parse_ms,
                              "rows_per_s": m / (parse_ms / 1e3), "text_GBps": m * text_per_row / (parse_ms / 1e3) / 1e9},
             "binary_pass_same_rows": {"ms": bin_ms, "rows_per_s": m / (bin_ms / 1e3),
                                       "GBps": m * bpr / (bin_ms / 1e3) / 1e9},
             "parse_over_binary_pass": parse_ms / bin_ms,
             "file_stream": {"ms": file_ms, "rows_per_s": n / (file_ms / 1e3),
                             "text_GBps": text_bytes / (file_ms / 1e3) / 1e9}}
    out = _base_line(args, world, METRIC, world * n / (file_ms / 1e3), file_ms, config,
                     {"bound": "host file read", "achieved": text_bytes / (file_ms / 1e3) / 1e9, "peak": None,
                      "unit": "GB/s", "frac": None, "traffic": None, "kernel": "csv_parse_kernel",
                      "algorithmic_bytes": text_bytes},
                     {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled (file pass)"]},
                     None, extra)
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.workload == "tables4096":
            run_tables(args, rank, world, local_rank)
        elif args.workload == "wide256":
            run_wide(args, rank, world, local_rank)
        elif args.workload == "f32table":
            run_f32table(args, rank, world, local_rank)
        elif args.workload == "table1_1e10":
            run_table1_stream(args, rank, world, local_rank)
        elif args.workload == "table1_file":
            run_table1_file(args, rank, world, local_rank)
        elif args.workload == "table1_csv":
            run_table1_csv(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
