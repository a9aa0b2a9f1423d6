"""Benchmark: harmonic summing + detection of the SKA-sized plane on GB300.

One step = one hs_run over the whole plane (85 templates x 2^21 bins, FP32,
H = 16 levels, 1e-8 false-alarm thresholds): every level sum of every point
is formed, tested and the candidates compacted.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--dtype f32|bf16] [--workload ska|small]

value      : points harmonic-summed per second (85 * 2^21 points per plane per
             step, all 16 levels), plane resident in HBM, whole job (all ranks).
e2e        : the same metric through hs_run_host with the plane in pinned host
             memory: host->device copy, summing, candidate read-back per step.
roofline   : the staged kernel's algorithmic bytes per launch (plane once +
             thresholds + candidate records) / its average launch duration
             (the timed region's CUDA-event time over its steps, launched
             back to back), against the measured HBM copy bandwidth.
cpu_baseline: the FP64 oracle on a bounded sample of the same plane, all host
             cores (threads over bin ranges).
--impl reference: the oracle alone, timed on the host cores (rank 0 only).

The default line also carries, each measured on its own after the main
measurement (skipped with --no-extras, and for every other workload):
precision  the same plane stored as BF16 and as FP16 (FP32 recheck copy):
           kernel time, throughput, roofline on its own bytes, records equal
           to the FP32 path's;
batch      64 beams log-uniform in [2^18, 2^22] bins packed in one plane, one
           summing launch per graph replay, against back-to-back hs_runs;
serve      the serving engine for 2 s of Poisson arrivals at 1000 beams/s:
           p50/p99 latency, then closed-loop capacity;
hfrac      the harmonic-fraction index map on the same plane: time per run,
           ratio to the stretch map, records in an oracle window (the oracle
           run in the CPU-baseline leg).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FOP points harmonic-summed/s (H=16) and effective HBM GB/s vs 8 TB/s"
UNIT = "points/s"
L2_BYTES = 129 * 2**20
ORDER_NAMES = {0: "53-step", 1: "linear", 2: "octave", 3: "semitone", 4: "53-step"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ska", choices=["ska", "small", "batch", "serve"])
    ap.add_argument("--shard", default="planes", choices=["planes", "band"],
                    help="N > 1: each rank sums its own plane (weak scaling), or one band "
                         "of the bins of the same plane (strong scaling)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="serve workload: length of the Poisson arrival phase")
    ap.add_argument("--serve-rate", type=float, default=1000.0, help="arrivals per second")
    ap.add_argument("--slots", type=int, default=16, help="serve workload: resident slots")
    ap.add_argument("--grid-per-sm", type=int, default=None,
                    help="resident CTAs per SM walking tiles (0: one CTA per tile); the batch "
                         "workload asks the autotuner when this is not given")
    ap.add_argument("--beams", type=int, default=64)
    ap.add_argument("--beam-log2", default="18,22",
                    help="batch workload: beam lengths log-uniform in [2^lo, 2^hi] bins")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--order", type=int, default=0)
    ap.add_argument("--tile-bins", type=int, default=0)
    ap.add_argument("--index", default="stretch", choices=["stretch", "hfrac"],
                    help="index map: the paper's stretch (Eq. 1-2) or harmonic fractions")
    ap.add_argument("--kernel", default="auto", choices=["auto", "staged", "generic"])
    ap.add_argument("--check-signs", action="store_true",
                    help="keep the staged kernel's per-value sign check (by default the plan "
                         "declares the plane non-negative: the synthetic planes are powers)")
    ap.add_argument("--stages", type=int, default=0,
                    help="staged kernel: ring stages of the pipelined variant (0: one CTA per tile)")
    ap.add_argument("--z-split", type=int, default=0,
                    help="pipelined variant: threads per bin (0 default)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU work of the oracle sample (core-seconds)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the precision, batch and serve sections "
                         "added to the line after the main measurement")
    return ap.parse_args()


def workload(name):
    from paper_1805_12258_gb300 import synth
    return synth.ska_plane(seed=1) if name == "ska" else synth.small_plane(seed=0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---- clocks ------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- CPU oracle leg --------------------------------------------------------------

def oracle_sample(plane, ta, H, cpu_seconds, threads, index="stretch"):
    """Time the FP64 oracle on all rows x a bin window; returns a dict."""
    import oracle
    oracle.build()
    idx = oracle.HFRAC if index == "hfrac" else oracle.STRETCH
    nt, n = plane.shape
    # calibrate: per-point cost on a small window, one thread
    cal = 2048
    t0 = time.perf_counter()
    oracle.detect(plane, H, ta, index=idx, f_lo=n // 2, f_hi=n // 2 + cal, threads=1)
    per_point = (time.perf_counter() - t0) / (nt * cal)
    # bins [n - bins, n): the high bins, whose reads span the plane
    bins = int(cpu_seconds / max(per_point, 1e-12) / nt)
    bins = max(min(n, threads * 64), min(bins, n))
    lo = n - bins
    t0 = time.perf_counter()
    cands, near = oracle.detect(plane, H, ta, index=idx, f_lo=lo, f_hi=n, threads=threads)
    dt = time.perf_counter() - t0
    what = "the whole plane" if bins == n else f"bins [{lo}, {n}) of the same plane"
    return {"value": nt * bins / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"all {nt} rows x {what} ({nt * bins} points, {H} levels, FP64), "
                      f"{threads} threads",
            "seconds": dt, "candidates_in_sample": int(len(cands)),
            "_window": (lo, n), "_records": cands, "_near": near}


def window_parity(gpu_records, cpu, rtol=1e-6):
    """The GPU run's records with bins inside the oracle sample's window
    against the oracle's records there: same (k, z, bin) set except points
    the oracle lists within 1e-5 of their threshold, powers within rtol."""
    lo, hi = cpu["_window"]
    r = gpu_records[(gpu_records["bin"] >= lo) & (gpu_records["bin"] < hi)]
    g = {(int(x["k"]), int(x["z"]), int(x["bin"])): float(x["power"]) for x in r}
    o = {(int(c["k"]), int(c["z"]), int(c["f"])): float(c["power"]) for c in cpu["_records"]}
    near = {(int(c["k"]), int(c["z"]), int(c["f"])) for c in cpu["_near"]}
    only_gpu = set(g) - set(o) - near
    only_oracle = set(o) - set(g) - near
    common = set(g) & set(o)
    err = max((abs(g[k] - o[k]) / max(abs(o[k]), 1e-30) for k in common), default=0.0)
    return {"window_bins": [int(lo), int(hi)], "gpu_records": len(r),
            "oracle_records": len(o), "near_threshold_excluded": len(near),
            "only_gpu": len(only_gpu), "only_oracle": len(only_oracle),
            "duplicates": len(r) - len(g), "max_rel_err": err, "rtol": rtol,
            "equal": (not only_gpu and not only_oracle and len(r) == len(g) and err <= rtol)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


KERNEL_SOURCES = ("hs_staged.cuh", "hs_device.cuh")


def source_hash(files):
    """Hash of the named csrc files' code with comments and white space
    removed, so comment edits keep a profile valid."""
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1805_12258_gb300", "csrc", f)) as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", "", code, flags=re.S)
        code = re.sub(r"//[^\n]*", "", code)
        h.update(re.sub(r"\s+", "", code).encode())
    return h.hexdigest()[:16]


def kernel_source_hash():
    """Hash of the staged kernel's code (hs_staged.cuh + hs_device.cuh)."""
    return source_hash(KERNEL_SOURCES)


def profiled_traffic(name):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(path) as fh:
            lines = [ln.split("|") for ln in fh if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    sha = kernel_source_hash()
    for parts in lines:
        parts = [x.strip() for x in parts]
        if len(parts) >= 3 and parts[0] == name and parts[2] == sha:
            return int(parts[1])
    return None


def profiled_instructions(name):
    """Warp instructions per run (ncu smsp__inst_executed.sum over the run's
    kernels) from profiles/instructions.txt, if taken on the current source of
    the files the entry names; else None."""
    path = os.path.join(ROOT, "profiles", "instructions.txt")
    try:
        with open(path) as fh:
            lines = [ln.split("|") for ln in fh if ln.strip() and not ln.startswith("#")]
    except OSError:
        return None
    for parts in lines:
        parts = [x.strip() for x in parts]
        if len(parts) >= 4 and parts[0] == name:
            try:
                if parts[2] == source_hash([f.strip() for f in parts[3].split(",")]):
                    return int(parts[1])
            except OSError:
                return None
    return None


def issue_roofline(instructions, us, clk, sms):
    """The instruction-issue roofline of a run: its warp instructions (ncu)
    over its measured time, against one warp instruction per cycle on each of
    the four schedulers of every SM at the SM clock sampled while it ran."""
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz")
    if not instructions or not mhz or not sms or us <= 0:
        return None
    achieved = instructions / (us / 1e6)
    peak = sms * 4 * mhz * 1e6
    return {"bound": "issue", "achieved": achieved, "peak": peak,
            "unit": "warp-instructions/s", "frac": achieved / peak,
            "instructions_per_run": instructions,
            "peak_from": f"{sms} SMs x 4 schedulers x 1 warp-instruction per cycle x "
                         f"{mhz:.0f} MHz (sampled)",
            "instructions_from": "profiles/instructions.txt (ncu smsp__inst_executed.sum)"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ---- reference arm: the oracle on the host cores ----------------------------------

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1805_12258_gb300 import synth
    oracle.build()
    wl = workload(args.workload)
    plane = synth.make_plane(wl)
    ta = synth.thresholds(wl.p_fa, wl.H, wl.n_templates)
    nt, n = plane.shape
    cores = host_cores()
    # size each step so the whole --warmup/--steps run takes about two minutes
    cal = 2048
    t0 = time.perf_counter()
    oracle.detect(plane, wl.H, ta, f_lo=n // 2, f_hi=n // 2 + cal, threads=1)
    per_point = (time.perf_counter() - t0) / (nt * cal)
    wall = min(8.0, 120.0 / max(1, args.steps + args.warmup))
    bins = int(wall * cores / max(per_point, 1e-12) / nt)
    bins = max(min(n, cores * 64), min(bins, n))
    lo = n - bins

    def step():
        t = time.perf_counter()
        oracle.detect(plane, wl.H, ta, f_lo=lo, f_hi=n, threads=cores)
        return nt * bins / (time.perf_counter() - t)

    for _ in range(args.warmup):
        step()
    vals = [step() for _ in range(args.steps)]
    v = statistics.median(vals)
    what = "all bins" if bins == n else f"bins [{lo}, {n})"
    sample = (f"all {nt} rows x {what} of the plane per step ({nt * bins} points, "
              f"{wl.H} levels, FP64), {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": nt * n / v * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl.name},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---- sections of the default line: the other forms ------------------------------------

def precision_summary(fop32, ta, H, ref_records, nonneg, steps=500):
    """The plane stored as BF16 and as FP16 (rounded on the device), summed
    with FP32 accumulation, levels near a threshold re-decided from the FP32
    copy; per storage: mean time per run (runs back to back, CUDA events
    around them), throughput, roofline on its own bytes, and whether its
    records equal the FP32 path's."""
    import torch

    from paper_1805_12258_gb300 import hs
    nt, n = fop32.shape
    stream = torch.cuda.current_stream()
    peak, kind = peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    out = {}
    for dt, tdt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        low = fop32.to(tdt)
        c = hs.CandBuffer(1 << 20)
        with hs.Plan(nt, n, H, ta, dtype=dt, assume_nonneg=nonneg) as plan:
            for _ in range(10):
                plan.run(low, c, stream, fop_f32=fop32)
            torch.cuda.synchronize()
            clocks = ClockSampler(torch.cuda.current_device())
            clocks.start()
            time.sleep(0.3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):  # back to back (summing and recheck kernels)
                plan.run(low, c, stream, fop_f32=fop32)
            e1.record(stream)
            torch.cuda.synchronize()
            clk = clocks.stop()
            recs, cnt, st = c.fetch(stream)
            name = (f"staged {nt}x{n} H={H} {dt} tb={plan.tile_bins} "
                    f"order={ORDER_NAMES[0]} with recheck")
        us = e0.elapsed_time(e1) / steps * 1e3
        algo = nt * n * 2 + H * nt * 4 + 16 * int(cnt) + 8
        out[dt] = {"storage": dt, "recheck": "FP32 copy", "mean_kernel_us": us,
                   "points_per_s": nt * n / (us / 1e6), "candidates": int(cnt),
                   "records_equal_fp32_path": bool(np.array_equal(recs, ref_records)),
                   "status": hs.hs_status_str(st),
                   "roofline": {"bound": "hbm", "achieved": algo / (us / 1e6) / 1e9,
                                "peak": peak, "unit": "GB/s",
                                "frac": algo / (us / 1e6) / 1e9 / peak,
                                "peak_kind": f"{kind} copy bandwidth",
                                "algo_bytes_per_launch": algo},
                   "issue_roofline": issue_roofline(profiled_instructions(name), us, clk, sms),
                   "clocks": clk}
        del low
    return out


def hfrac_summary(fop32, ta, H, stretch_us, steps=20):
    """The harmonic-fraction index map (level k sums the terms h/k, h = 1..k)
    on the same plane: its staged kernels' mean time per run (runs back to
    back, CUDA events around them; one launch per level family), throughput,
    the ratio to the stretch map's kernel time, and its records (returned
    beside the summary)."""
    import torch

    from paper_1805_12258_gb300 import hs
    nt, n = fop32.shape
    stream = torch.cuda.current_stream()
    peak, kind = peaks()
    c = hs.CandBuffer(1 << 20)
    with hs.Plan(nt, n, H, ta, index="hfrac") as plan:
        for _ in range(3):
            plan.run(fop32, c, stream)
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):  # back to back
            plan.run(fop32, c, stream)
        e1.record(stream)
        launches = hs.hs_last_launch_count()
        torch.cuda.synchronize()
        clk = clocks.stop()
        recs, cnt, st = c.fetch(stream)
        kernel, tb = plan.kernel, plan.tile_bins
    us = e0.elapsed_time(e1) / steps * 1e3
    algo = nt * n * 4 + H * nt * 4 + 16 * int(cnt) + 8
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    name = f"{kernel} hfrac {nt}x{n} H={H} f32 tb={tb}"
    return {"index": "hfrac", "kernel": kernel, "tile_bins": tb, "launches_per_run": launches,
            "mean_us_per_run": us, "points_per_s": nt * n / (us / 1e6),
            "level_sums_per_s": nt * n * H / (us / 1e6), "time_vs_stretch_map": us / stretch_us,
            "candidates": int(cnt), "status": hs.hs_status_str(st),
            "effective_hbm_gbs": algo / (us / 1e6) / 1e9,
            "frac_of_peak_on_unique_bytes": algo / (us / 1e6) / 1e9 / peak,
            "peak_kind": f"{kind} copy bandwidth",
            "issue_roofline": issue_roofline(profiled_instructions(name), us, clk, sms),
            "clocks": clk}, recs


# ---- our arm ------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1805_12258_gb300 import build as hsbuild
    from paper_1805_12258_gb300 import hs, shard, synth

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    hsbuild.build()

    wl = workload(args.workload)
    band = args.shard == "band" and ws > 1
    if rank and not band:
        wl.seed = shard.rank_seed(wl.seed, rank)  # each rank sums its own plane
    nt, n, H = wl.n_templates, wl.n_bins, wl.H
    es = 4 if args.dtype == "f32" else 2
    host32 = torch.empty((nt, n), dtype=torch.float32, pin_memory=True)
    synth.make_plane(wl, out=host32.numpy())
    plane_np = host32.numpy()
    ta = synth.thresholds(wl.p_fa, H, nt)
    if args.dtype == "f32":
        host = host32
    else:
        lowp = torch.bfloat16 if args.dtype == "bf16" else torch.float16
        host = host32.to(lowp).pin_memory()
    fop = host.cuda()
    fop32 = fop if args.dtype == "f32" else host32.cuda()
    # the plan declares the plane non-negative unless --check-signs: verify
    # that promise on the whole plane (outside the timed region)
    nonneg_verified = bool((fop32 >= 0).all().item())
    cands = hs.CandBuffer(1 << 20)
    plan = hs.Plan(nt, n, H, ta, dtype=args.dtype, order=args.order, tile_bins=args.tile_bins,
                   grid_per_sm=args.grid_per_sm or 0, stages=args.stages, z_split=args.z_split,
                   index=args.index, kernel=args.kernel, assume_nonneg=not args.check_signs)
    stream = torch.cuda.current_stream()

    f_lo, f_hi = shard.band_bounds(n, ws, plan.tile_bins)[rank] if band else (0, n)

    def step():
        f32 = None if args.dtype == "f32" else fop32
        if band:
            plan.run_range(fop, cands, f_lo, f_hi, stream, fop_f32=f32)
        else:
            plan.run(fop, cands, stream, fop_f32=f32)

    for _ in range(max(3, args.warmup)):
        step()
    st, n_cand = cands.sync(stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    # a plane smaller than L2 is timed cold: 512 MB of scratch is written
    # before every launch and the throughput comes from the launches' own
    # CUDA-event times (the scratch writes stay outside them).  Otherwise the
    # launches run back to back with no event between them (a pair of events
    # per launch costs about 4 us of a 146 us step), and the average launch
    # duration is the timed region's elapsed time over the steps.
    cold = nt * n * es < L2_BYTES
    plan.set_timing(cold)
    plan.kernel_time()  # clear
    clocks.start()
    time.sleep(0.3)  # sampler warm-up
    scratch = torch.empty(512 << 20, dtype=torch.uint8, device="cuda") if cold else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches_before = 0
    # the timed region: a barrier over the ranks and a device synchronize on
    # each side of exactly args.steps steps
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(args.steps):
        if cold:
            scratch.fill_(i & 0xff)
        step()
        launches_before += hs.hs_last_launch_count()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = e0.elapsed_time(e1)
    kern_ms, kern_n = plan.kernel_time() if cold else (elapsed_ms, args.steps)
    plan.set_timing(True)
    hot_us = None
    per_launch_event_us = None
    if not cold:  # for reference: the same launches, each inside its own event pair
        plan.kernel_time()
        for _ in range(min(args.steps, 200)):
            step()
        torch.cuda.synchronize()
        pk, pn = plan.kernel_time()
        per_launch_event_us = pk / max(pn, 1) * 1e3
    if cold:  # the same launches back to back, plane resident in L2
        plan.kernel_time()
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        hk, hn = plan.kernel_time()
        hot_us = hk / max(hn, 1) * 1e3
        elapsed_ms = kern_ms
        del scratch
    # 20 single launches, each after a 512 MB scratch write (L2 flushed):
    # best and median of the launches' own event times
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    single = []
    for i in range(20):
        flush.fill_(i & 0xff)
        plan.kernel_time()
        step()
        single.append(plan.kernel_time()[0] * 1e3)
    del flush
    cold_launch = {"best_us": min(single), "median_us": float(np.median(single)), "n": 20,
                   "l2": "512 MB scratch written before each launch"}
    plan.set_timing(False)
    t = torch.tensor([elapsed_ms], device="cuda")
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    elapsed_ms = float(t.item())
    st, n_cand = cands.sync(stream)
    timed_records = cands.fetch(stream)[0]  # the last timed launch's records

    precision = None
    if args.dtype != "f32":
        # candidate set of the 16-bit plane (with FP32 rechecks) against the
        # FP32 path on the FP32 copy: equal record for record by design
        low = timed_records
        c32 = hs.CandBuffer(1 << 20)
        with hs.Plan(nt, n, H, ta, index=args.index, kernel=args.kernel) as p32:
            p32.run(fop32, c32, stream)
            r32 = c32.fetch(stream)[0]
        precision = {"storage": args.dtype, "recheck": "FP32 copy",
                     "candidates": int(len(low)), "fp32_path_candidates": int(len(r32)),
                     "records_equal_fp32_path": bool(np.array_equal(low, r32))}

    points = nt * n
    # whole-job points per step: every rank's plane, or the one banded plane
    value = points * (1 if band else ws) * args.steps / (elapsed_ms / 1e3)
    ms_per_step = elapsed_ms / args.steps
    mean_kernel_s = kern_ms / max(kern_n, 1) / 1e3
    algo_bytes = nt * (f_hi - f_lo) * es + H * nt * 4 + 16 * n_cand + 8
    if args.dtype != "f32":
        algo_bytes += 0  # rechecks read only near-threshold points of the FP32 copy
    peak, peak_kind = peaks()
    achieved_gbs = algo_bytes / mean_kernel_s / 1e9
    kname = (f"staged {nt}x{n} H={H} {args.dtype} tb={plan.tile_bins} "
             f"order={ORDER_NAMES.get(args.order, args.order)}"
             if plan.kernel == "staged" else f"generic {nt}x{n} H={H} {args.dtype} {args.index}")
    if args.index == "hfrac" and plan.kernel == "staged":
        kname = (f"staged hfrac {nt}x{n} H={H} {args.dtype} tb={plan.tile_bins} "
                 "(one launch per level family; time per run)")

    # e2e through hs_run_host: pinned host plane -> device, sum, records -> host
    e2e = None
    if args.e2e_steps > 0 and not band:  # the host path sums whole planes
        dev = torch.empty_like(host, device="cuda")
        out = np.zeros(1 << 16, hs.CAND_DTYPE)
        # 16-bit planes: only the 16-bit plane crosses the host link in bulk;
        # the rechecks read the page-locked FP32 copy in place
        h32 = None if args.dtype == "f32" else host32
        plan.run_host(host, dev, cands, out, stream, fop32_host=h32)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.e2e_steps):
            _, ne = plan.run_host(host, dev, cands, out, stream, fop32_host=h32)
            d2h += 8 + 16 * min(ne, len(out))
        te = time.perf_counter() - t0
        tt = torch.tensor([te], device="cuda")
        if ws > 1:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        te = float(tt.item())
        e2e = {"value": points * ws * args.e2e_steps / te, "unit": UNIT,
               "h2d_bytes_per_step": nt * n * es, "d2h_bytes_per_step": d2h // args.e2e_steps,
               "ms_per_step": te * 1e3 / args.e2e_steps,
               "e2e_candidates_equal_device_run": bool(ne == n_cand)}
        if h32 is not None:
            e2e["recheck"] = "FP32 copy read in place from page-locked host memory"
        del dev

    extras = (rank == 0 and ws == 1 and not args.no_extras and args.workload == "ska" and
              args.dtype == "f32" and args.index == "stretch" and not band)
    cpu, parity, cpu_hfrac = None, None, None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_sample(plane_np, ta, H, args.cpu_seconds, host_cores(), index=args.index)
        if not band:
            parity = window_parity(timed_records, cpu)
        cpu = {k: v for k, v in cpu.items() if not k.startswith("_")}
        if extras:  # a short oracle window for the harmonic-fraction section
            cpu_hfrac = oracle_sample(plane_np, ta, H, 3.0, host_cores(), index="hfrac")

    sections = {}
    if extras:
        # the other forms of the method, each measured on its own after the
        # main measurement: 16-bit storage of this plane, the 64-beam batch,
        # a short serving run
        sections["precision"] = precision_summary(fop, ta, H, timed_records,
                                                  not args.check_signs)
        sections["batch"] = batch_summary(args, steps=20, tune=False)
        torch.cuda.empty_cache()
        sections["serve"] = serve_summary(args, seconds=2.0, rate=1000.0, closed_k=1000)
        torch.cuda.empty_cache()
        hf, hf_recs = hfrac_summary(fop, ta, H, mean_kernel_s * 1e6)
        if cpu_hfrac is not None:
            hf["parity_window"] = window_parity(hf_recs, cpu_hfrac)
            hf["parity_in_window"] = hf["parity_window"]["equal"]
            hf["cpu_oracle_points_per_s"] = cpu_hfrac["value"]
        sections["hfrac"] = hf
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong" if band else "weak", "vs_baseline": None, "dtype": args.dtype,
            "data": "synthetic",
            "config": {"workload": wl.name, "n_templates": nt, "n_bins": n, "H": H,
                       "p_fa": wl.p_fa, "kernel": plan.kernel, "index": args.index,
                       "inputs": ("checked for negative values" if args.check_signs else
                                  "declared non-negative (powers; plan option assume_nonneg)"),
                       "inputs_verified_nonneg": nonneg_verified,
                       "tile_bins": plan.tile_bins,
                       "order": args.order, "grid_per_sm": args.grid_per_sm or 0,
                       "candidates": n_cand,
                       "l2": (f"plane {nt * n * es / 1e6:.1f} MB < {L2_BYTES / 1e6:.0f} MB L2: "
                              "512 MB scratch written before every launch (cold); time = the "
                              "launches' own event times" if cold else
                              f"plane {nt * n * es / 1e6:.0f} MB > {L2_BYTES / 1e6:.0f} MB L2: "
                              "inputs larger than L2, no flush"),
                       "hot_l2_kernel_us": hot_us,
                       "single_launch_after_l2_flush": cold_launch,
                       "parallelism": (f"one plane in {ws} frequency bands (bins "
                                       f"[{f_lo}, {f_hi}) on rank 0)" if band else
                                       f"{ws} independent planes (one per GPU)")},
            "level_sums_per_s": value * H,
            "effective_hbm_gbs": algo_bytes * ws * args.steps / (elapsed_ms / 1e3) / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": peak,
                         "unit": "GB/s", "frac": achieved_gbs / peak,
                         "traffic": profiled_traffic(kname),
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "kernel": kname, "algo_bytes_per_launch": algo_bytes,
                         "mean_kernel_us": mean_kernel_s * 1e6,
                         "duration_from": ("each launch's own event pair" if cold else
                                           "timed region elapsed / steps (launches back "
                                           "to back, counter reset included)"),
                         "per_launch_event_us": per_launch_event_us,
                         "frac_of_8tbs": algo_bytes / mean_kernel_s / 8e12},
            "precision": precision if precision is not None else sections.get("precision"),
            "batch": sections.get("batch"),
            "serve": sections.get("serve"),
            "hfrac": sections.get("hfrac"),
            "parity_in_window": None if parity is None else parity["equal"],
            "parity_window": parity,
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
            "gpu_launches": launches_before, "status": hs.hs_status_str(st),
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        dist.destroy_process_group()


def packed_beams(nt, sizes, seed):
    """Beams of the given lengths side by side along the bins of one device
    plane (offsets a multiple of 4 bins = 16 bytes), Exponential(1) noise
    drawn on the device; returns (plane, offsets)."""
    import torch
    offs, at = [], 0
    for n in sizes:
        offs.append(at)
        at = (at + n + 3) // 4 * 4
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    plane = torch.empty((nt, at), device="cuda").exponential_(generator=g)
    return plane, offs


def batch_summary(args, *, n_beams=64, lo=18.0, hi=22.0, steps=20, tune=False):
    """64 beams of 85 templates x n_bins (log-uniform in [2^lo, 2^hi], seed
    3), H = 16, FP32, packed side by side in one plane and summed by one
    graph replay per step (a counter reset and one summing launch); the same
    beams as one hs_run each, back to back, are timed beside it and their
    records compared.  tune: the autotuner picks the launch form (packed, or
    launches carrying each beam's descriptors), tile order and grid."""
    import torch

    from paper_1805_12258_gb300 import autotune, hs, synth
    nt, H = 85, 16
    sizes = [int(x) for x in synth.beam_lengths(n_beams, seed=3, lo_log2=lo, hi_log2=hi)]
    ta = synth.thresholds(1e-8, H, nt)
    plane, offs = packed_beams(nt, sizes, seed=3000)
    pitch = plane.shape[1]
    bufs = [hs.CandBuffer(1 << 16) for _ in sizes]
    beams = [(plane[:, o:], n, cb) for o, n, cb in zip(offs, sizes, bufs)]
    nonneg = not args.check_signs
    choice, table = {"form": "packed", "order": 0, "grid_per_sm": 0}, None
    if tune:
        choice, table = autotune.tune_batch(nt, H, ta, beams, assume_nonneg=nonneg,
                                            packed=(plane, offs))
    points = nt * sum(sizes)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with hs.Batch(nt, H, ta, grid_per_sm=choice["grid_per_sm"], max_beams=len(sizes),
                  order=choice["order"], assume_nonneg=nonneg) as batch:
        if choice["form"] == "packed":
            batch.set_packed(plane, [(o, n, cb) for o, n, cb in zip(offs, sizes, bufs)])
        else:
            batch.set_beams(beams)
        for _ in range(max(3, args.warmup)):
            batch.graph_run(stream)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        time.sleep(0.3)
        e0.record(stream)
        for _ in range(steps):
            batch.graph_run(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1) / steps
        rec_batch = [cb.fetch(stream)[0] for cb in bufs]
        tiles, launches = batch.tiles, batch.launches
    # the same beams one hs_run each, back to back on the stream
    seq_bufs = [hs.CandBuffer(1 << 16) for _ in sizes]
    plans = [hs.Plan(nt, n, H, ta, row_pitch=pitch, assume_nonneg=nonneg) for n in sizes]
    try:
        def sequential():
            for plan, o, cb in zip(plans, offs, seq_bufs):
                plan.run(plane[:, o:], cb, stream=stream)
        for _ in range(3):
            sequential()
        torch.cuda.synchronize()
        seq_steps = max(3, min(steps, 10))
        e0.record(stream)
        for _ in range(seq_steps):
            sequential()
        e1.record(stream)
        torch.cuda.synchronize()
        t_seq = e0.elapsed_time(e1) / seq_steps
        rec_seq = [cb.fetch(stream)[0] for cb in seq_bufs]
    finally:
        for plan in plans:
            plan.close()
    n_cand = int(sum(len(r) for r in rec_batch))
    algo = nt * sum(sizes) * 4 + H * nt * 4 + 16 * n_cand + 8 * len(sizes)
    peak, kind = peaks()
    del plane, beams
    return {
        "workload": f"batch of {len(sizes)} beams, 85 templates x n_bins log-uniform in "
                    f"[2^{lo:g}, 2^{hi:g}], H=16 fp32",
        "beams": len(sizes), "bins_total": sum(sizes), "tiles": tiles,
        "form": choice["form"], "tile_order": ORDER_NAMES.get(choice["order"], choice["order"]),
        "grid_per_sm": choice["grid_per_sm"],
        "launches_per_step": 1 + launches, "graph": True, "ms_per_step": ms,
        "points_per_s": points / (ms / 1e3), "candidates": n_cand,
        "sequential_hs_run_ms": t_seq, "speedup_vs_sequential": t_seq / ms,
        "records_equal_per_plane_runs": all(np.array_equal(a, b)
                                            for a, b in zip(rec_batch, rec_seq)),
        "inputs": "checked for negative values" if args.check_signs else
                  "declared non-negative (powers)",
        "roofline": {"bound": "hbm", "achieved": algo / (ms / 1e3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": algo / (ms / 1e3) / 1e9 / peak,
                     "peak_kind": f"{kind} copy bandwidth", "algo_bytes_per_step": algo,
                     "frac_of_8tbs": algo / (ms / 1e3) / 8e12},
        "timed": "CUDA events around the graph replays (counter reset + summing launches)",
        "autotune": table, "clocks": clk,
    }


def run_batch(args):
    """The batch workload as its own line (see batch_summary)."""
    import torch

    from paper_1805_12258_gb300 import build as hsbuild
    torch.cuda.set_device(0)
    hsbuild.build()
    lo, hi = (float(x) for x in args.beam_log2.split(","))
    tune = args.grid_per_sm is None or args.grid_per_sm < 0
    steps = max(3, min(args.steps, 200))
    b = batch_summary(args, n_beams=args.beams, lo=lo, hi=hi, steps=steps, tune=tune)
    print(json.dumps({
        "metric": METRIC, "value": b["points_per_s"], "unit": UNIT, "n_gpus": 1,
        "steps": steps, "warmup": args.warmup, "ms_per_step": b["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (planes generated on the device)",
        "config": {k: v for k, v in b.items() if k not in ("roofline", "clocks", "autotune")},
        "roofline": b["roofline"], "autotune": b["autotune"], "e2e": None,
        "cpu_baseline": None, "clocks": b["clocks"],
        "gpu_launches": b["launches_per_step"] * steps,
    }), flush=True)


def serve_summary(args, seconds, rate, closed_k=None):
    """The serving engine under Poisson arrivals (seed 4, `rate` beams/s for
    `seconds`) of beams with 85 templates x n_bins log-uniform in
    [2^18, 2^22], H = 16, FP32 or BF16 (50/50), 0-10 injected signals each;
    then closed-loop phases that keep the queue full to measure the engine's
    capacity, with planes generated per request and with planes already
    resident.  Returns a summary dict."""
    import threading

    import numpy as np
    import torch

    from paper_1805_12258_gb300 import hs, synth

    nt, H = 85, 16
    ta = synth.thresholds(1e-8, H, nt)
    rng = np.random.Generator(np.random.Philox(4))
    lo, hi = (float(x) for x in args.beam_log2.split(","))

    def draw(k):
        n = np.rint(2.0 ** rng.uniform(lo, hi, size=k)).astype(np.int64)
        dt = np.where(rng.random(k) < 0.5, "bf16", "f32")
        sig = rng.integers(0, 11, size=k)
        return n, dt, sig

    n_max = int(round(2.0 ** hi))
    with hs.Server(nt, H, ta, n_slots=args.slots, slot_bins=n_max, cand_capacity=4096,
                   queue_limit=1 << 16, assume_nonneg=not args.check_signs) as srv:
        # warm-up: every path once (allocations, first launches)
        wn, wd, ws = draw(2 * args.slots)
        warm = [srv.submit(10**6 + i, int(wn[i]), str(wd[i]), int(ws[i])) for i in range(len(wn))]
        for t in warm:
            srv.wait(t)

        def phase(n_bins, dts, sigs, arrivals, seed0):
            """Submit at the arrival times (None: as fast as admission
            allows); a second thread collects results in submit order."""
            results, tickets, rejected = [], [], [0]
            done = threading.Event()

            def collect():
                i = 0
                while True:
                    if i < len(tickets):
                        out = srv.wait(tickets[i])
                        results.append(out[0])
                        i += 1
                    elif done.is_set():
                        return
                    else:
                        time.sleep(0.0002)

            th = threading.Thread(target=collect)
            th.start()
            t0 = time.perf_counter()
            for i in range(len(n_bins)):
                if arrivals is not None:
                    dt = t0 + arrivals[i] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                while True:
                    t = srv.submit(seed0 + i, int(n_bins[i]), str(dts[i]), int(sigs[i]))
                    if t is not None:
                        tickets.append(t)
                        break
                    if arrivals is not None:
                        rejected[0] += 1
                        break
                    time.sleep(0.0002)  # closed loop: wait for room
            done.set()
            th.join()
            return results, rejected[0]

        # open loop: Poisson arrivals
        k = int(rate * seconds * 1.2) + 16
        gaps = rng.exponential(1.0 / rate, size=k)
        arr = np.cumsum(gaps)
        k = int(np.searchsorted(arr, seconds))
        n_bins, dts, sigs = draw(k)
        clocks = ClockSampler(0)
        clocks.start()
        res_open, rej = phase(n_bins, dts, sigs, arr[:k], 2 * 10**6)
        # closed loop: queue kept full for capacity
        kc = closed_k or max(64, int(rate * 3))
        cn, cd, cs = draw(kc)
        res_closed, _ = phase(cn, cd, cs, None, 3 * 10**6)
        # closed loop over planes already resident (made upstream beforehand):
        # the engine's own capacity, without the plane generator
        pool = []
        pn, pd, _ = draw(16)
        for i in range(16):
            n = int(pn[i])
            ld = (n + 7) // 8 * 8
            f32 = torch.empty((nt, ld), dtype=torch.float32, device="cuda")
            if pd[i] == "f32":
                hs.hs_synth_fop(f32, None, "f32", nt, n, ld, 5 * 10**6 + i, 5)
                pool.append((n, "f32", f32, None))
            else:
                b16 = torch.empty((nt, ld), dtype=torch.bfloat16, device="cuda")
                hs.hs_synth_fop(b16, f32, "bf16", nt, n, ld, 5 * 10**6 + i, 5)
                pool.append((n, "bf16", b16, f32))
        torch.cuda.synchronize()
        kr = closed_k or max(64, int(rate * 3))
        res_res, rtickets = [], []
        done_r = threading.Event()

        def collect_r():
            i = 0
            while True:
                if i < len(rtickets):
                    res_res.append(srv.wait(rtickets[i])[0])
                    i += 1
                elif done_r.is_set():
                    return
                else:
                    time.sleep(0.0002)

        thr = threading.Thread(target=collect_r)
        thr.start()
        rn = []
        for i in range(kr):
            n, dt, fop, f32 = pool[i % len(pool)]
            while True:
                t = srv.submit(0, n, dt, 0, fop=fop, fop32=f32)
                if t is not None:
                    rtickets.append(t)
                    rn.append(n)
                    break
                time.sleep(0.0002)
        done_r.set()
        thr.join()
        del pool
        clk = clocks.stop()
        st = srv.stats()

    def summary(results, n_bins):
        lat = np.array([(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r in results])
        svc = np.array([(r["t_done_ns"] - r["t_admit_ns"]) / 1e6 for r in results])
        span = (max(r["t_done_ns"] for r in results) - min(r["t_submit_ns"] for r in results)) / 1e9
        pts = nt * int(np.sum(n_bins[:len(results)]))
        bad = {"overflow": sum(r["status"] == hs.HS_ERR_OVERFLOW for r in results),
               "other": sum(r["status"] not in (hs.HS_OK, hs.HS_ERR_OVERFLOW) for r in results)}
        return {"requests": len(results), "failed": bad,
                "latency_ms": {"p50": float(np.percentile(lat, 50)),
                               "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
                "service_ms": {"p50": float(np.percentile(svc, 50)),
                               "p99": float(np.percentile(svc, 99))},
                "points_per_s": pts / span, "seconds": span,
                "mean_group": float(np.mean([r["group_size"] for r in results]))}

    so, sc = summary(res_open, n_bins), summary(res_closed, cn)
    sr = summary(res_res, np.array(rn))
    # the plane generator alone (the upstream stand-in each request pays for)
    gen = {}
    ld = (n_max + 7) // 8 * 8
    f32 = torch.empty((nt, ld), dtype=torch.float32, device="cuda")
    b16 = torch.empty((nt, ld), dtype=torch.bfloat16, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name in ("f32", "bf16"):
        for rep in range(4):
            e0.record()
            hs.hs_synth_fop(f32 if name == "f32" else b16, None if name == "f32" else f32, name,
                            nt, n_max, ld, 99 + rep, 10)
            e1.record()
            torch.cuda.synchronize()
        gen[name] = e0.elapsed_time(e1)
    del f32, b16
    return {
        "workload": f"serving: Poisson {rate:g} beams/s for {seconds:g} s, 85 templates x "
                    f"n_bins log-uniform in [2^{lo:g}, 2^{hi:g}], H=16, FP32/BF16 50/50, "
                    "0-10 signals",
        "slots": args.slots,
        "inputs": "checked for negative values" if args.check_signs else
                  "declared non-negative (powers)",
        "open_loop": dict(so, rejected=rej, offered_per_s=rate),
        "closed_loop": sc,
        "closed_loop_resident_planes": dict(sr, note="planes made beforehand and kept "
                                            "resident; requests sum them in place"),
        "latency": "steady clock from hs_server_submit to the candidates in host memory "
                   "(service: from admission into a slot)",
        "generator_ms_per_2^22_plane": gen, "stats": st, "clocks": clk,
    }


def run_serve(args):
    """The serving workload as its own line (see serve_summary)."""
    import torch

    from paper_1805_12258_gb300 import build as hsbuild
    torch.cuda.set_device(0)
    hsbuild.build()
    sv = serve_summary(args, args.serve_seconds, args.serve_rate)
    print(json.dumps({
        "metric": "FOP points harmonic-summed/s served (planes resident, queue kept full)",
        "value": sv["closed_loop_resident_planes"]["points_per_s"], "unit": UNIT, "n_gpus": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
        "data": "synthetic (planes generated on the device per request)",
        "config": {"workload": sv["workload"], "slots": sv["slots"],
                   "l2": "inputs larger than L2", "inputs": sv["inputs"]},
        **{k: sv[k] for k in ("open_loop", "closed_loop", "closed_loop_resident_planes",
                              "latency", "generator_ms_per_2^22_plane", "stats", "clocks")},
        "e2e": None, "cpu_baseline": None,
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
