"""Benchmark of the mapping-driven re-layout path on GB300.

One step = one pass over every re-layout row of the hot path, each on its
full-size synthetic workload, through the C ABI (``llgb_copy``/``pack``/
``unpack``):

  C3  512x512x512 CFD records {rho,u,v,w,e: f32, flag: i16, id: u16}, u32
      index type, static inner extents:
        AoS -> SoA(mb), SoA(mb) -> AoS, SoA(mb) -> AoSoA32,
        AoSoA32 -> SoA(mb), AoSoA8 -> AoSoA32
  C1  2^26 INT6 records {a..d: u32, e,f: i32}, b in {1, 3, 7, 12, 17, 31}
      (values drawn for each b): SoA(mb) -> BitpackIntSoA (pack) and back
  C2  2^25 MIXED_F records {x,y,z: f64, w: f32}, N(0, 1e3):
        SoA(mb) -> BitpackFloatSoA(E, M) and back for E in {5, 8, 11},
        M in {2, 10, 23, 52}; SoA(mb) -> Bytesplit(SoA);
        SoA(mb) -> ChangeType(f64->f32, SoA)

value = algorithmic bytes (every source blob byte read + every destination
blob byte written) of the step / device time of the step, in GB/s.  Every
input is larger than L2, so no flush is needed between steps.  The n-body
consumer (65,536 particles) is timed in its own loop and reported under
"nbody"; "sweeps" holds the Split / Null and bit-packed AoSoA rows and the
small 65,536-particle case (warm and cold L2).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs the whole per-GPU workload on its own GPU (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "re-layout GB/s (read+write) vs HBM peak"
PROFILE = os.path.join(ROOT, "profiles", "copy_kernel_relayout_suite.md")


# ------------------------------------------------------------ workload --

def rows_spec(only=None, scale=1):
    """(name, config, source mapping, destination mapping) of every row: the
    C3 re-layout pairs; C1 pack and unpack at every width b; C2 pack and
    unpack in every (E, M) format, Bytesplit and ChangeType.  `only` keeps
    rows whose name contains it; `scale` divides the record counts (for small
    profiling captures)."""
    from paper_2302_08251_gb300 import synth
    c3 = dict(name="C3", record=synth.CFD, n=512 ** 3 // scale, ext=(512 // scale, 512, 512), itype="u32",
              static=(False, True, True), fields="cfd")
    c2 = dict(name="C2", record=synth.MIXED_F, n=(1 << 25) // scale, ext=((1 << 25) // scale,), itype="u32",
              static=None, fields="mixed_f")
    soa = {"kind": "soa_mb"}
    aos = {"kind": "aos"}
    a32 = {"kind": "aosoa", "lanes": 32}
    a8 = {"kind": "aosoa", "lanes": 8}
    rows = [
        ("C3 AoS->SoA", c3, aos, soa),
        ("C3 SoA->AoS", c3, soa, aos),
        ("C3 SoA->AoSoA32", c3, soa, a32),
        ("C3 AoSoA32->SoA", c3, a32, soa),
        ("C3 AoSoA8->AoSoA32", c3, a8, a32),
    ]
    for b in C1_BITS:
        # values are drawn in [0, 2^b) and [-2^(b-1), 2^(b-1)): a source per width
        c1 = dict(name=f"C1b{b}", record=synth.INT6, n=(1 << 26) // scale, ext=((1 << 26) // scale,), itype="u32",
                  static=None, fields="int6", bits=b)
        bp = {"kind": "bitpack_int", "bits": b}
        rows += [(f"C1 pack b={b}", c1, soa, bp), (f"C1 unpack b={b}", c1, bp, soa)]
    for e, m in C2_FORMATS:
        bf = {"kind": "bitpack_float", "exp": e, "man": m}
        rows += [(f"C2 pack E{e}M{m}", c2, soa, bf), (f"C2 unpack E{e}M{m}", c2, bf, soa)]
    rows += [
        ("C2 bytesplit", c2, soa, {"kind": "bytesplit", "inner": soa}),
        ("C2 changetype f64->f32", c2, soa, {"kind": "changetype", "ct": [("f64", "f32")], "inner": soa}),
    ]
    return [r for r in rows if only is None or only in r[0]]


C1_BITS = (1, 3, 7, 12, 17, 31)
C2_FORMATS = tuple((e, m) for e in (5, 8, 11) for m in (2, 10, 23, 52))


def key(m):
    return json.dumps(m, sort_keys=True)


class Workload:
    """Device views for every row; sources are seeded and resident in HBM."""

    def __init__(self, device, seed, only=None, scale=1):
        import torch
        from paper_2302_08251_gb300 import llgb, synth
        self.rows = []
        self.records = {}
        cache = {}  # (config name, mapping) -> source view
        for name, cfg, src_map, dst_map in rows_spec(only, scale):
            cname = cfg["name"]
            rec = self.records.setdefault(cname, llgb.Record(cfg["record"]))
            kw = dict(index_type=cfg["itype"], static=cfg["static"])
            base_key = (cname, key({"kind": "soa_mb"}))
            if base_key not in cache:
                fields = synth.device_fields(cfg["fields"], cfg["n"], seed, device=device, bits=cfg.get("bits", 12))
                blobs = [f.contiguous().view(torch.uint8) for f in fields]
                cache[base_key] = llgb.View(rec, {"kind": "soa_mb"}, cfg["ext"], blobs=blobs, **kw)
            src_key = (cname, key(src_map))
            if src_key not in cache:
                v = llgb.View(rec, src_map, cfg["ext"], **kw)
                llgb.llgb_copy(cache[base_key], v)
                cache[src_key] = v
            src = cache[src_key]
            dst = llgb.View(rec, dst_map, cfg["ext"], **kw)
            nbytes = sum(src.blob_sizes) + sum(dst.blob_sizes)
            self.rows.append(dict(name=name, cfg=cfg, src=src, dst=dst, bytes=nbytes,
                                  src_map=src_map, dst_map=dst_map))
        torch.cuda.synchronize()
        self.bytes = sum(r["bytes"] for r in self.rows)

    def step(self, stream, events=None):
        from paper_2302_08251_gb300 import llgb
        for k, r in enumerate(self.rows):
            if events is not None:
                events[k][0].record(stream)
            llgb.llgb_copy(r["src"], r["dst"], stream)
            if events is not None:
                events[k][1].record(stream)


# -------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during timing."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
             "clocks.mem,clocks.max.mem,temperature.gpu")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mem, temp, smax, mmax, reasons = [], [], [], None, None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
            try:
                mem.append(float(parts[9]))
                mmax = float(parts[10])
                temp.append(float(parts[11]))
            except (IndexError, ValueError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "mem_mhz": statistics.median(mem) if mem else None, "mem_max_mhz": mmax,
                "gpu_temp_c": statistics.median(temp) if temp else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- helpers --

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    # the kernels, and the planner and launch shapes that decide what they run
    for f in ("copy_kernel.cuh", "copy.cu", "copy_mode0.cu", "copy_mode1.cu", "copy_mode3.cu", "copy_gather.cu",
              "stream_loops.cuh", "stream_specs.h", "fconv.cuh", "job.h", "plan.cpp", "capi.cpp"):
        with open(os.path.join(ROOT, "paper_2302_08251_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """Per-step DRAM traffic of the copy kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    got = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            got[k.strip()] = v.strip()
    if got.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(got["dram_bytes_per_step"])
    except (KeyError, ValueError):
        return None


def max_over_ranks(ms, world):
    """The slowest rank's time: what the whole job waited for (all-reduce
    MAX over the process group; the value itself when world == 1)."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_rank, world, ms_per_step):
    """Whole-job GB/s: every rank moves bytes_per_rank per step (weak
    scaling), and the step lasts as long as the slowest rank."""
    return bytes_per_rank * world / (ms_per_step * 1e-3) / 1e9


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------- CPU oracle --

def oracle_copy_threaded(src, dst, threads):
    """The oracle's copy over record ranges on `threads` host threads (ctypes
    releases the GIL).  Ranges start at multiples of 1024 records, so no two
    threads share a bit-stream word or an AoSoA block."""
    from concurrent.futures import ThreadPoolExecutor
    n = src.n
    step = max(1024, (n + threads - 1) // threads // 1024 * 1024)
    ranges = [(i, min(n, i + step)) for i in range(0, n, step)]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda r: src.copy_to(dst, r[0], r[1]), ranges))


def oracle_sample(seconds_budget=12.0, seed=1, threads=None):
    """Time the oracle copy on a bounded sample of every row: the first
    records of each workload, sized so the whole single-thread sample takes
    ~10-30 s; the same sample is then timed on all host cores.  Returns
    (single-thread GB/s, all-cores GB/s, threads, sample, single-thread s)."""
    import numpy as np
    import oracle
    from paper_2302_08251_gb300 import synth
    oracle.build()
    threads = threads or os.cpu_count() or 1
    total_bytes, total_time, total_mt, parts = 0, 0.0, 0.0, []
    per_row = seconds_budget / len(rows_spec())
    for name, cfg, src_map, dst_map in rows_spec():
        m = 4096
        while True:
            rec = cfg["record"]
            if cfg["fields"] == "int6":
                fields = synth.int6(m, cfg.get("bits", 12), seed)
            elif cfg["fields"] == "mixed_f":
                fields = synth.mixed_f(m, seed)
            else:
                fields = synth.cfd(m, seed)
            base = oracle.OracleView(rec, {"kind": "soa_mb"}, m)
            for f, col in enumerate(fields):
                u = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[col.itemsize]
                base.set_field_values(f, col.view(u).astype(np.uint64))
            src = oracle.OracleView(rec, src_map, m)
            base.copy_to(src)
            dst = oracle.OracleView(rec, dst_map, m)
            t0 = time.perf_counter()
            src.copy_to(dst)
            dt = time.perf_counter() - t0
            if dt * 4 > per_row or m >= cfg["n"]:
                break
            m *= 4
        dst_mt = oracle.OracleView(rec, dst_map, m)
        t0 = time.perf_counter()
        oracle_copy_threaded(src, dst_mt, threads)
        dt_mt = time.perf_counter() - t0
        nbytes = sum(src.blob_sizes) + sum(dst.blob_sizes)
        total_bytes += nbytes
        total_time += dt
        total_mt += dt_mt
        parts.append(f"{name}: {m} records")
    return (total_bytes / total_time / 1e9, total_bytes / total_mt / 1e9, threads, "; ".join(parts),
            total_time)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample(seconds_budget=2.0)
    vals, singles, times, sample, threads = [], [], [], "", 1
    for _ in range(args.steps):
        v1, v, threads, sample, t = oracle_sample(seconds_budget=8.0)
        vals.append(v)
        singles.append(v1)
        times.append(t)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(times) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bytes/int/f64",
            "data": "synthetic (seeded)",
            "config": {"workload": "llama re-layout suite, 43 rows (C1 all widths, C2 all formats, "
                                   "bytesplit, changetype, C3 512^3 pairs), bounded sample",
                       "parallelism": "host threads over record ranges"},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "single_thread_value": statistics.median(singles), "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- main --

def run_gpu(args):
    import torch
    from paper_2302_08251_gb300 import build, llgb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("gloo")
    build.build()
    llgb.lib()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    wl = Workload(device, seed=2302082510 + rank, only=args.only, scale=args.scale)
    stream = torch.cuda.current_stream()
    nrows = len(wl.rows)
    for _ in range(args.warmup):
        wl.step(stream)
    barrier()

    events = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(nrows)]
              for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        wl.step(stream, events[s])
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = [[events[s][k][0].elapsed_time(events[s][k][1]) for k in range(nrows)]
                 for s in range(args.steps)]
    total_ms = max_over_ranks(total_ms, world)
    ms_per_step = total_ms / args.steps
    value = job_throughput(wl.bytes, world, ms_per_step)

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    kernel_ms = sum(sum(x) for x in launch_ms) / args.steps
    achieved = wl.bytes / (kernel_ms * 1e-3) / 1e9
    rows_out = {}
    for k, r in enumerate(wl.rows):
        ms = statistics.median(launch_ms[s][k] for s in range(args.steps))
        gbs = r["bytes"] / (ms * 1e-3) / 1e9
        rows_out[r["name"]] = {"bytes": r["bytes"], "ms": round(ms, 4), "GB/s": round(gbs, 1),
                               "frac": round(gbs / hbm, 4)}
    traffic = profiled_traffic()

    # end to end through host buffers (first among the extras: it measured
    # 179-269 GB/s after the n-body leg, 255-262 GB/s on its own)
    e2e = e2e_bench(wl, stream, args) if rank == 0 and not args.no_extras else None
    # n-body consumer (65,536 particles through AoS / SoA / AoSoA32 views)
    nbody = nbody_bench(device, args) if rank == 0 and not args.no_extras else None
    batched = serving = sweeps = None
    step_bytes = wl.bytes
    if rank == 0 and not args.no_extras:
        del wl
        torch.cuda.empty_cache()
        batched = batched_bench(device, args)
        torch.cuda.empty_cache()
        serving = serving_bench(device, args)
        torch.cuda.empty_cache()
        sweeps = sweeps_bench(device)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bytes/int/f64->f32", "data": "synthetic (seeded), resident in HBM",
            "config": {"workload": "llama re-layout suite, 43 rows: C3 512^3 CFD AoS<->SoA, SoA<->AoSoA32, "
                                   "AoSoA8->AoSoA32 (u32, static inner extents); C1 2^26 INT6 "
                                   "BitpackInt pack+unpack at b=1,3,7,12,17,31; C2 2^25 MIXED_F "
                                   "BitpackFloat pack+unpack at E=5,8,11 x M=2,10,23,52, Bytesplit, "
                                   "ChangeType f64->f32",
                       "bytes_per_step": step_bytes, "l2": "inputs > L2 (no flush needed)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "traffic": traffic,
                         "per": "step (one launch per row; achieved and traffic both per step)",
                         "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                         "kernel": "llgb::copy_kernel", "spec_frac_8tbs": round(achieved / 8000.0, 4)},
            "rows": rows_out,
            "clocks": clk,
            "gpu_launches": nrows * args.steps,
            "e2e": e2e,
            "nbody": nbody,
            "batched": batched,
            "serving": serving,
            "sweeps": sweeps,
        }
        if not args.no_cpu_baseline and not args.no_extras:
            v1, v, threads, sample, _ = oracle_sample()
            line["cpu_baseline"] = {"value": round(v, 4), "unit": "GB/s", "cores": threads,
                                    "kind": "oracle", "single_thread_value": round(v1, 4),
                                    "sample": sample}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def nbody_bench(device, args):
    import torch
    from paper_2302_08251_gb300 import llgb, synth
    rec = llgb.Record(synth.PARTICLE)
    n = 65536
    fields = synth.device_fields("particle", n, 7, device=device)
    base = llgb.View(rec, {"kind": "soa_mb"}, (n,), blobs=[f.view(torch.uint8) for f in fields])
    out = {}
    for name, m in (("AoS", {"kind": "aos"}), ("SoA", {"kind": "soa_mb"}),
                    ("AoSoA32", {"kind": "aosoa", "lanes": 32})):
        v = llgb.View(rec, m, (n,))
        llgb.llgb_copy(base, v)
        for _ in range(2):
            llgb.llgb_nbody_step(v, 0.01, 1e-4)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(3, args.steps)
        a.record()
        for _ in range(reps):
            llgb.llgb_nbody_step(v, 0.01, 1e-4)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        flops = 20.0 * n * n
        out[name] = {"ms_per_step": round(ms, 4), "TFLOP/s": round(flops / (ms * 1e-3) / 1e12, 2)}
    roofline = nbody_roofline(device, base, rec, n)
    instrumented = nbody_instrumentation_bench(device, base, rec, n, args)
    traversal = nbody_traversal_bench(device, base, rec, n)
    return {"n": n, "flop_per_interaction": 20, "views": out, "instrumented": instrumented,
            "traversal": traversal, "roofline": roofline}


def nbody_roofline(device, base, rec, n, seconds=1.0):
    """The n-body update is FP32-ALU-bound: its TFLOP/s against the FP32 FMA
    throughput probe (llgb_fma_probe, 2 FLOP per FMA), each run for about
    `seconds` with nvidia-smi sampling the SM clock, so that both are stated
    at the clock they ran at."""
    import torch
    from paper_2302_08251_gb300 import llgb
    sink = torch.zeros(1, dtype=torch.float32, device=device)
    gpu = device.index if device.index is not None else 0

    def timed_loop(fn, seconds):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        reps = max(3, int(seconds / max(a.elapsed_time(b) * 1e-3, 1e-6)))
        clk = ClockSampler(gpu)
        clk.start()
        time.sleep(0.3)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, clk.stop()

    fmas = []
    probe_ms, probe_clk = timed_loop(lambda: fmas.append(llgb.llgb_fma_probe(100000, sink)), seconds)
    peak = 2.0 * fmas[-1] / (probe_ms * 1e-3) / 1e12
    v = llgb.View(rec, {"kind": "soa_mb"}, (n,))
    llgb.llgb_copy(base, v)
    step_ms, step_clk = timed_loop(lambda: llgb.llgb_nbody_step(v, 0.01, 1e-4), seconds)
    achieved = 20.0 * n * n / (step_ms * 1e-3) / 1e12
    out = {"bound": "alu", "achieved": round(achieved, 2), "peak": round(peak, 2), "unit": "TFLOP/s",
           "frac": round(achieved / peak, 4), "view": "SoA",
           "peak_source": "FP32 FMA throughput probe (llgb_fma_probe), measured in this run",
           "sm_mhz": {"nbody": step_clk.get("sm_mhz"), "probe": probe_clk.get("sm_mhz")},
           "reasons": sorted(set(step_clk.get("reasons", [])) | set(probe_clk.get("reasons", []))),
           "nominal_peak_max_clock": round(152 * 128 * 2 * 2.07e9 / 1e12, 1)}
    if step_clk.get("sm_mhz") and probe_clk.get("sm_mhz"):
        out["frac_at_equal_clock"] = round(achieved / peak * probe_clk["sm_mhz"] / step_clk["sm_mhz"], 4)
    return out


TRAVERSAL_VIEWS = [("AoS", {"kind": "aos"}), ("SoA", {"kind": "soa_mb"}),
                   ("AoSoA8", {"kind": "aosoa", "lanes": 8}), ("AoSoA32", {"kind": "aosoa", "lanes": 32}),
                   ("AoSoA48", {"kind": "aosoa", "lanes": 48}), ("AoSoA3", {"kind": "aosoa", "lanes": 3})]


def nbody_traversal_bench(device, base, rec, n_update, n_move=1 << 26):
    """Index against blocks traversal (Sec. 5): the move phase alone on 2^26
    particles (1.9 GB views, larger than L2; algorithmic bytes 36 per
    particle: pos and vel read, pos written) and the update phase alone on
    the 65,536-particle system, per mapping."""
    import torch
    from paper_2302_08251_gb300 import llgb, synth
    peaks, _ = measured_peaks()
    hbm = float(peaks["hbm_gbs"])

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    move = {}
    fields = synth.device_fields("particle", n_move, 19, device=device)
    big = llgb.View(rec, {"kind": "soa_mb"}, (n_move,), blobs=[f.view(torch.uint8) for f in fields])
    for name, m in TRAVERSAL_VIEWS:
        v = llgb.View(rec, m, (n_move,))
        llgb.llgb_copy(big, v)
        row = {}
        for trav in ("index", "blocks"):
            ms = timed(lambda: llgb.llgb_nbody_move(v, 1e-4, trav), 10)
            g = 36.0 * n_move / (ms * 1e-3) / 1e9
            row[trav] = {"ms": round(ms, 4), "GB/s": round(g, 1), "frac": round(g / hbm, 4)}
        move[name] = row
        del v
        torch.cuda.empty_cache()
    del big, fields
    torch.cuda.empty_cache()
    update = {}
    for name, m in TRAVERSAL_VIEWS:
        v = llgb.View(rec, m, (n_update,))
        llgb.llgb_copy(base, v)
        update[name] = {trav: {"ms": round(timed(lambda: llgb.llgb_nbody_update(v, 0.01, 1e-4, trav), 5), 4)}
                        for trav in ("index", "blocks")}
    return {"move": {"n": n_move, "bytes_per_particle": 36, "views": move},
            "update": {"n": n_update, "views": update}}


def nbody_instrumentation_bench(device, base, rec, n, args):
    """FieldAccessCount / Heatmap (Sec. 4) on the SoA n-body step: step time
    with each instrumentation against the plain step, and counter memory
    against the view's bytes."""
    import torch
    from paper_2302_08251_gb300 import llgb
    v = llgb.View(rec, {"kind": "soa_mb"}, (n,))
    llgb.llgb_copy(base, v)
    counts = torch.zeros(14, dtype=torch.int64, device=device)
    heats = {g: torch.zeros(llgb.llgb_heatmap_counters(v, g), dtype=torch.int64, device=device)
             for g in (1, 64)}
    variants = {
        "plain": lambda: llgb.llgb_nbody_step(v, 0.01, 1e-4),
        "FieldAccessCount, atomic per access": lambda: llgb.llgb_nbody_step_instrumented(
            v, 0.01, 1e-4, field_counts=counts, count_mode="atomic"),
        "FieldAccessCount, per-CTA counters": lambda: llgb.llgb_nbody_step_instrumented(
            v, 0.01, 1e-4, field_counts=counts, count_mode="block"),
        "Heatmap, 64-byte granules": lambda: llgb.llgb_nbody_step_instrumented(
            v, 0.01, 1e-4, heat=heats[64], granularity=64),
        "Heatmap, bytes": lambda: llgb.llgb_nbody_step_instrumented(v, 0.01, 1e-4, heat=heats[1], granularity=1),
    }
    out = {}
    for name, fn in variants.items():
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        out[name] = {"ms_per_step": round(a.elapsed_time(b) / reps, 4)}
    plain = out["plain"]["ms_per_step"]
    view_bytes = sum(llgb.blob_sizes(rec, {"kind": "soa_mb"}, (n,)))
    for name in out:
        out[name]["slowdown"] = round(out[name]["ms_per_step"] / plain, 3)
    out["FieldAccessCount, atomic per access"]["counter_bytes"] = 14 * 8
    out["FieldAccessCount, per-CTA counters"]["counter_bytes"] = 14 * 8
    for g, key in ((64, "Heatmap, 64-byte granules"), (1, "Heatmap, bytes")):
        out[key]["counter_bytes"] = heats[g].numel() * 8
        out[key]["memory_overhead"] = round(heats[g].numel() * 8 / view_bytes, 3)
    return out


def time_copy(src, dst, reps=10):
    """Median device ms of `reps` single copies (CUDA events per launch)."""
    import torch
    from paper_2302_08251_gb300 import llgb
    llgb.llgb_copy(src, dst)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        llgb.llgb_copy(src, dst)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


SPLIT_ROWS = [
    # (row name, record kind, source mapping, destination mapping)
    ("2^26 INT6 AoS -> Split{a,b,c,d: BitpackInt b=12 | e,f: SoA-MB}", "int6", {"kind": "aos"},
     {"kind": "split", "fields": [0, 1, 2, 3], "inner": {"kind": "bitpack_int", "bits": 12},
      "rest": {"kind": "soa_mb"}}),
    ("2^26 particles AoS -> Split{pos: SoA-MB | vel, mass: AoSoA32}", "particle", {"kind": "aos"},
     {"kind": "split", "fields": [0, 1, 2], "inner": {"kind": "soa_mb"},
      "rest": {"kind": "aosoa", "lanes": 32}}),
    ("2^26 particles AoS -> Split{mass: Null | rest: SoA-MB}", "particle", {"kind": "aos"},
     {"kind": "split", "fields": [6], "inner": {"kind": "null"}, "rest": {"kind": "soa_mb"}}),
]


def split_rows(device, entry):
    """Copies into and out of Split views (Sec. 3): each row's forward copy
    and the copy back into the source's mapping, algorithmic bytes = source
    blobs + destination blobs."""
    import torch
    from paper_2302_08251_gb300 import llgb, synth
    n = 1 << 26
    rows = {}
    for name, kind, src_map, dst_map in SPLIT_ROWS:
        leaves = {"int6": synth.INT6, "particle": synth.PARTICLE}[kind]
        rec = llgb.Record(leaves)
        fields = synth.device_fields(kind, n, 23, device=device)
        soa = llgb.View(rec, {"kind": "soa_mb"}, (n,), blobs=[f.view(torch.uint8) for f in fields])
        src = llgb.View(rec, src_map, (n,))
        llgb.llgb_copy(soa, src)
        del soa, fields
        dst = llgb.View(rec, dst_map, (n,))
        nbytes = sum(llgb.blob_sizes(rec, src_map, (n,))) + sum(llgb.blob_sizes(rec, dst_map, (n,)))
        rows[name] = {"forward": entry(nbytes, time_copy(src, dst)), "back": entry(nbytes, time_copy(dst, src))}
        del src, dst
        torch.cuda.empty_cache()
    return rows


def bitpack_aosoa_rows(device, entry):
    """Bit-packed mappings organised as AoSoA (L lanes) against the SoA
    organisation, packed from and unpacked to SoA multi-blob: 2^26 INT6
    records at b = 12, 2^25 MIXED_F records at E8M23."""
    import torch
    from paper_2302_08251_gb300 import llgb, synth
    soa = {"kind": "soa_mb"}
    rows = {}
    for label, kind, n, rec_leaves, mp in (
            ("INT6 b=12", "int6", 1 << 26, synth.INT6, {"kind": "bitpack_int", "bits": 12}),
            ("MIXED_F E8M23", "mixed_f", 1 << 25, synth.MIXED_F, {"kind": "bitpack_float", "exp": 8, "man": 23})):
        rec = llgb.Record(rec_leaves)
        fields = synth.device_fields(kind, n, 29, device=device)
        base = llgb.View(rec, soa, (n,), blobs=[f.contiguous().view(torch.uint8) for f in fields])
        plain = llgb.View(rec, soa, (n,))
        for org, m in (("SoA", mp), ("AoSoA32", dict(mp, lanes=32)), ("AoSoA256", dict(mp, lanes=256))):
            packed = llgb.View(rec, m, (n,))
            nbytes = sum(llgb.blob_sizes(rec, soa, (n,))) + sum(llgb.blob_sizes(rec, m, (n,)))
            rows[f"{label} {org}"] = {"pack": entry(nbytes, time_copy(base, packed)),
                                      "unpack": entry(nbytes, time_copy(packed, plain))}
            del packed
            torch.cuda.empty_cache()
        del fields, base, plain
        torch.cuda.empty_cache()
    return rows


def sweeps_bench(device):
    """Rows beyond the configurations' step: copies into and out of Split /
    Null views (2^26 records); the bit-packed AoSoA organisation against SoA;
    and the small C0 case (65,536 particles AoS -> SoA multi-blob), whose 3.7 MB
    fit L2: its time is reported warm (copies back to back), with L2 flushed
    before a single copy, and as the host's submission cost per call."""
    import torch
    from paper_2302_08251_gb300 import llgb, synth
    peaks, _ = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    out = {}
    soa = {"kind": "soa_mb"}

    def entry(nbytes, ms):
        g = nbytes / (ms * 1e-3) / 1e9
        return {"ms": round(ms, 4), "GB/s": round(g, 1), "frac": round(g / hbm, 4)}

    out["F2 Split / Null"] = split_rows(device, entry)
    out["F3 bit-packed AoSoA organisation"] = bitpack_aosoa_rows(device, entry)

    n = 65536
    rec = llgb.Record(synth.PARTICLE)
    fields = synth.device_fields("particle", n, 3, device=device)
    base = llgb.View(rec, soa, (n,), blobs=[f.view(torch.uint8) for f in fields])
    aos = llgb.View(rec, {"kind": "aos"}, (n,))
    llgb.llgb_copy(base, aos)
    dst = llgb.View(rec, soa, (n,))
    nbytes = 2 * 28 * n
    # warm: 50 copies back to back between two events (host submission
    # overlaps the GPU; one event pair per copy would also time the ~7 us it
    # takes the host to plan from the cache and launch); host: that
    # submission cost per call on the CPU clock
    llgb.llgb_copy(aos, dst)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    a.record()
    for _ in range(50):
        llgb.llgb_copy(aos, dst)
    b.record()
    host_us = (time.perf_counter() - t0) / 50 * 1e6
    b.synchronize()
    warm = a.elapsed_time(b) / 50
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)  # > L2
    cold = []
    for _ in range(30):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        llgb.llgb_copy(aos, dst)
        b.record()
        b.synchronize()
        cold.append(a.elapsed_time(b))
    cold_ms = statistics.median(cold)
    out["C0 AoS -> SoA-MB, 65,536 particles (3.7 MB)"] = {
        "warm_us": round(warm * 1e3, 2), "host_us_per_call": round(host_us, 2),
        "cold_l2_us": round(cold_ms * 1e3, 2),
        "cold_l2_GB/s": round(nbytes / (cold_ms * 1e-3) / 1e9, 1)}
    return out


def batched_bench(device, args, chunk_bytes=24 * (1 << 30)):
    """All 4,096 config-4 requests (log-uniform record counts, mixed mapping
    pairs), in arrival order, in chunks of at most ~24 GB of algorithmic
    bytes: one launch per view (llgb_copy each) against one batched launch
    replayed from a CUDA graph, with identical bytes checked on the device.
    Before timing, llgb_autotune tunes each mapping pair once on its largest
    request; batch entries take those shapes."""
    import torch
    from paper_2302_08251_gb300 import llgb, serve
    reqs = serve.workload(count=4096)
    ex = serve.GpuExecutor(streams=1, seed=11)
    chunks, cur, cur_bytes = [], [], 0
    for r in reqs:
        nb = ex.nbytes(r)
        if cur and cur_bytes + nb > chunk_bytes:
            chunks.append(cur)
            cur, cur_bytes = [], 0
        cur.append(r)
        cur_bytes += nb
    if cur:
        chunks.append(cur)
    stream = torch.cuda.current_stream()
    reps = max(2, min(args.steps, 3))

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # tune each mapping pair once, on its largest request
    llgb.llgb_autotune_clear()
    largest = {}
    for r in reqs:
        k = (tuple(r.record), json.dumps(r.src_map, sort_keys=True), json.dumps(r.dst_map, sort_keys=True))
        if k not in largest or r.n > largest[k].n:
            largest[k] = r
    tuned = {}
    for k, r in largest.items():
        ex.allocate(r)
        src, dst, _ = r.views
        cfg = llgb.llgb_autotune(src, dst, stream)
        tuned[f"{r.record[0][0]}: {r.src_map['kind']} -> {r.dst_map['kind']}"] = dict(cfg, n=r.n)
        ex.release(r)
        r.views = None
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    total_bytes, ms_view, ms_batch, same, launches = 0, 0.0, 0.0, True, 0
    for chunk in chunks:
        pairs, alt, nbytes = [], [], 0
        for r in chunk:
            ex.allocate(r)
            src, dst, _ = r.views
            pairs.append((src, dst))
            alt.append(llgb.View(ex._record(r.record), r.dst_map, (r.n,)))
            nbytes += ex.nbytes(r)
        torch.cuda.synchronize()

        def per_view():
            for (src, _), d in zip(pairs, alt):
                llgb.llgb_copy(src, d, stream)
        batch = llgb.Batch(pairs)
        ms_view += timed(per_view)
        ms_batch += timed(lambda: batch.launch(stream, use_graph=True))
        same = same and all(torch.equal(x, y) for (_, d), a in zip(pairs, alt) for x, y in zip(d.blobs, a.blobs))
        launches = max(launches, batch.info()["launches"])
        batch.close()
        total_bytes += nbytes
        del pairs, alt, batch
        for r in chunk:
            r.views = None
        torch.cuda.empty_cache()
    peaks, _ = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    gbs = total_bytes / ms_batch / 1e6
    return {"requests": len(reqs), "chunks": len(chunks), "bytes": total_bytes,
            "kernel_launches_batched_max": launches, "autotuned": tuned,
            "per_view": {"ms": round(ms_view, 3), "GB/s": round(total_bytes / ms_view / 1e6, 1),
                         "launches": len(reqs)},
            "batched_graph": {"ms": round(ms_batch, 3), "GB/s": round(gbs, 1), "frac": round(gbs / hbm, 4)},
            "speedup": round(ms_view / ms_batch, 3), "identical_bytes": bool(same)}


def serving_bench(device, args):
    """The continuous-batching request loop on the config-4 stream: 4,096
    requests, Poisson arrivals at 2,000 req/s, 64 GB HBM budget, 4 streams."""
    from paper_2302_08251_gb300 import serve
    reqs = serve.workload(count=4096)
    ex = serve.GpuExecutor(streams=4, seed=12)
    ex.warm([(r.record, r.src_map, r.dst_map) for r in reqs])  # gather programs, before the clock starts
    srv = serve.Server(ex, budget_bytes=64 * serve.GB, deadline_s=60.0)
    stats = srv.run(reqs)
    out = stats.summary()
    out["arrival_rate_hz"] = 2000.0
    out["budget_GB"] = 64
    return out


def e2e_bench(wl, stream, args):
    """The same step through host buffers: every row's source blobs go
    host->device from pinned memory, the copy runs, the destination blobs
    come back device->host, all inside the timed region.  Copies in and out
    run on streams of their own, ordered by events: every row copies its
    inputs into device blobs of its own (rows that share a source view on the
    device get a view each, so that no copy-in waits for another row's
    re-layout), a row's copy-in waits for the previous step's re-layout of
    that row, its re-layout for its copy-in and for the previous step's
    copy-out of its destination, and its copy-out for its re-layout -- so
    copies in run ahead while copies out follow, both directions of the
    full-duplex host link busy at once."""
    import torch
    from paper_2302_08251_gb300 import llgb
    hosts, seen, dev_src = {}, set(), []
    for r in wl.rows:
        sid = id(r["src"])
        if sid not in hosts:
            hosts[sid] = [torch.empty(b.numel(), dtype=torch.uint8, pin_memory=True)
                          for b in r["src"].blobs]
            for h, b in zip(hosts[sid], r["src"].blobs):
                h.copy_(b)
        if sid in seen:
            cfg = r["cfg"]
            dev_src.append(llgb.View(wl.records[cfg["name"]], r["src_map"], cfg["ext"],
                                     index_type=cfg["itype"], static=cfg["static"]))
        else:
            seen.add(sid)
            dev_src.append(r["src"])
    out_max = max(max(b.numel() for b in r["dst"].blobs) for r in wl.rows)
    host_out = torch.empty(out_max, dtype=torch.uint8, pin_memory=True)  # copy-outs run in order on one stream
    h2d = sum(sum(b.numel() for b in r["src"].blobs) for r in wl.rows)
    d2h = sum(sum(b.numel() for b in r["dst"].blobs) for r in wl.rows)
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    K = len(wl.rows)
    ev_in = [torch.cuda.Event() for _ in range(K)]
    ev_kern = [torch.cuda.Event() for _ in range(K)]
    ev_out = [torch.cuda.Event() for _ in range(K)]
    for k in range(K):  # recorded once, so that the first step's waits are satisfied
        ev_kern[k].record(stream)
        ev_out[k].record(stream)

    def step():
        for k, r in enumerate(wl.rows):
            s_in.wait_event(ev_kern[k])  # the previous step's re-layout of this row read these blobs
            with torch.cuda.stream(s_in):
                for h, b in zip(hosts[id(r["src"])], dev_src[k].blobs):
                    b.copy_(h, non_blocking=True)
            ev_in[k].record(s_in)
            stream.wait_event(ev_in[k])
            stream.wait_event(ev_out[k])
            llgb.llgb_copy(dev_src[k], r["dst"], stream)
            ev_kern[k].record(stream)
            s_out.wait_event(ev_kern[k])
            with torch.cuda.stream(s_out):
                for b in r["dst"].blobs:
                    host_out[:b.numel()].copy_(b, non_blocking=True)
            ev_out[k].record(s_out)

    step()
    torch.cuda.synchronize()
    reps = max(1, min(args.steps, 3))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s_in.wait_event(a)
    s_out.wait_event(a)
    for _ in range(reps):
        step()
    stream.wait_stream(s_in)
    stream.wait_stream(s_out)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    link = host_link_rates(hosts, wl, host_out, s_in, s_out)
    return {"value": round(wl.bytes / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(ms, 3),
            "steps": reps, "overlap": "copies in run ahead on one stream, copies out follow on another",
            "host_link_GBs": link,
            "transfer_frac_of_link": round((h2d + d2h) / (ms * 1e-3) / 1e9 / link["both"], 4)}


def host_link_rates(hosts, wl, host_out, s_in, s_out):
    """Copy rates of the host link from the e2e leg's own pinned buffers: one
    source blob in, a destination blob out, and both at once (GB/s)."""
    import torch
    src_h, src_d = max(((h, b) for r in wl.rows for h, b in zip(hosts[id(r["src"])], r["src"].blobs)),
                       key=lambda hb: hb[0].numel())
    dst_d = max((b for r in wl.rows for b in r["dst"].blobs), key=lambda b: b.numel())
    nb = min(src_h.numel(), dst_d.numel(), host_out.numel())

    def timed(h2d, d2h):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s_in.wait_event(a)
        s_out.wait_event(a)
        if h2d:
            with torch.cuda.stream(s_in):
                src_d[:nb].copy_(src_h[:nb], non_blocking=True)
        if d2h:
            with torch.cuda.stream(s_out):
                host_out[:nb].copy_(dst_d[:nb], non_blocking=True)
        cur = torch.cuda.current_stream()
        cur.wait_stream(s_in)
        cur.wait_stream(s_out)
        b.record()
        b.synchronize()
        return nb * (int(h2d) + int(d2h)) / (a.elapsed_time(b) * 1e-3) / 1e9

    return {k: round(max(timed(*f) for _ in range(3)), 1)
            for k, f in (("h2d", (True, False)), ("d2h", (False, True)), ("both", (True, True)))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the n-body, e2e and CPU-baseline legs (profiling runs)")
    ap.add_argument("--only", default=None, help="run only rows whose name contains this")
    ap.add_argument("--scale", type=int, default=1, help="divide record counts (profiling)")
    ap.add_argument("--nbody-only", action="store_true",
                    help="run only W + K n-body steps on 65,536 SoA particles (profiling)")
    ap.add_argument("--batch-only", type=int, default=0, metavar="N",
                    help="run only one batch of the first N serving-workload requests of at most "
                         "3e6 records, W + K launches (profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.nbody_only:
        return run_nbody_only(args)
    if args.batch_only:
        return run_batch_only(args)
    return run_gpu(args)


def run_batch_only(args):
    """One llgb_batch of the first N requests (of at most 3e6 records) of the
    serving workload, launched W + K times, for profiling the batch kernel;
    prints the batch's size and the mean time of the K timed launches."""
    import torch
    from paper_2302_08251_gb300 import llgb, serve
    reqs = [r for r in serve.workload(count=4096) if r.n <= 3_000_000][:args.batch_only]
    ex = serve.GpuExecutor(streams=1, seed=11)
    pairs, nbytes = [], 0
    for r in reqs:
        ex.allocate(r)
        src, dst, _ = r.views
        pairs.append((src, dst))
        nbytes += ex.nbytes(r)
    batch = llgb.Batch(pairs)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.launch(stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        batch.launch(stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / max(1, args.steps)
    assert llgb.llgb_device_status(reset=True) == 0
    print(json.dumps({"batch_entries": len(pairs), "bytes": nbytes, "info": batch.info(),
                      "ms_per_launch": round(ms, 4), "GB/s": round(nbytes / ms / 1e6, 1)}))
    return 0


def run_nbody_only(args):
    """W + K plain n-body steps on 65,536 particles through a SoA view, for
    profiling the update and move kernels; prints the mean step time."""
    import torch
    from paper_2302_08251_gb300 import llgb, synth
    n = 65536
    rec = llgb.Record(synth.PARTICLE)
    fields = synth.device_fields("particle", n, 7, device="cuda")
    v = llgb.View(rec, {"kind": "soa_mb"}, (n,), blobs=[f.view(torch.uint8) for f in fields])
    for _ in range(args.warmup):
        llgb.llgb_nbody_step(v, 0.01, 1e-4)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        llgb.llgb_nbody_step(v, 0.01, 1e-4)
    b.record()
    torch.cuda.synchronize()
    print(json.dumps({"nbody_ms_per_step": round(a.elapsed_time(b) / max(1, args.steps), 4), "n": n}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
