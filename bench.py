#!/usr/bin/env python3
"""Benchmark: batched complex-to-complex FFT throughput on one GB300 (or N replicas).

Workload (one step): the plain-method sweep - forward and inverse c2c
complex64 transforms for N = 2^3 .. 2^12 with batch = 2^26 / N, i.e. 20
out-of-place calls over the same 512 MiB synthetic input (SplitMix64 uniform
[-1, 1)), each moving 2^30 algorithmic bytes (16 bytes per complex point: one
read, one write).  Inputs are larger than L2, so no flush is needed between
calls.

Printed (rank 0, one JSON line): whole-job GB/s over the timed steps, the
live roofline of the dominant kernel (CUDA events on its launch stream), the
end-to-end figure through gbfft_execute_host (host buffers, copies inside the
timed region), the clocks sampled during the timed region, and the FP64
oracle timed on the host cores as a CPU baseline.

``--impl reference`` times the FP64 CPU oracle instead (the reference arm):
same metric and unit, each step a bounded sample of the same workload.

Multi-GPU: ``--gpus N`` under torchrun runs N independent replicas (the
transform batch shards by rows with no exchange); barrier + max-over-ranks
timing; value = bytes of all ranks / slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Batched C2C FFT GB/s (% HBM peak) vs plain; serving p50/p99 at stated rel. error"
UNIT = "GB/s"
SWEEP = [1 << k for k in range(3, 13)]
TOTAL = 1 << 26            # complex elements per call
BYTES_PER_CALL = 16 * TOTAL  # algorithmic bytes: 8 read + 8 written per complex
WORKLOAD = ("plain-method sweep: forward+inverse c2c complex64, N=2^3..2^12, "
            "batch=2^26/N (512 MiB in + 512 MiB out per call), uniform[-1,1)")
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gbfft", "reference"], default="gbfft")
    ap.add_argument("--config", choices=["sweep", "pr1", "mixed", "twopass", "tc", "ragged", "serving", "f64", "nd", "pease"],
                    default="sweep",
                    help="sweep (default, the headline line) or one of the other configurations")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the short live runs of the two-pass, tensor-core, ragged and serving paths")
    ap.add_argument("--sizes", type=str, default=None,
                    help="comma-separated subset of the sweep (for small profiling cases)")
    ap.add_argument("--dtype", type=int, default=0,
                    help="plan dtype for the sweep runner (0 FP32, 1 FP16x2 and 2 BF16x2 tensor-core; profiling)")
    ap.add_argument("--variant", type=int, default=None,
                    help="plan variant for the sweep runner (tensor-core dtypes: 0 mma.sync, 1 tcgen05; profiling)")
    ap.add_argument("--ragged-graph-only", action="store_true",
                    help="ragged config: time only the single persistent launch (for profiling)")
    ap.add_argument("--points-log2", type=int, default=26,
                    help="complex points per call (default 26: the 512 MiB sweep workload)")
    args = ap.parse_args()
    global SWEEP, TOTAL, BYTES_PER_CALL
    if args.sizes:
        SWEEP = [int(v) for v in args.sizes.split(",")]
    TOTAL = 1 << args.points_log2
    BYTES_PER_CALL = 16 * TOTAL
    return args


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


# Files that define the single-pass rows kernels (the sweep's dominant kernel):
# a recorded DRAM-traffic figure is valid only while these hash the same.
ROWS_KERNEL_SOURCES = ("codelets.cuh", "stockham.cuh", "variants.cuh", "rows_pow2.cu")


def source_digest(files=ROWS_KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2207_06803_gb300", "csrc")
    for name in files:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = source_digest()
    with open(path) as f:
        for line in f:
            parts = line.split("#")[0].split()
            if len(parts) == 3 and parts[0] == kernel_key and parts[2] == digest:
                return float(parts[1])
    return None


class ClockSampler:
    """nvidia-smi sampling (200 ms) during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_index: int):
        self.samples = []
        self.proc = None
        self.device_index = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        for p in self.samples:
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, p[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# --------------------------------------------------------------------------

def oracle_sweep_once(flat, points_per_call: int, nthreads: int) -> float:
    """Run the FP64 oracle (recursive radix-2) over `points_per_call` points of
    every (N, direction) of the sweep; return wall seconds."""
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    for n in SWEEP:
        rows = max(1, points_per_call // n)
        x = flat[: rows * n].reshape(rows, n).astype(np.complex128)
        for sign in (oracle.FORWARD, oracle.INVERSE):
            oracle.fft_radix2(x, sign, nthreads)
    return time.perf_counter() - t0


def calibrate_oracle(flat, nthreads: int, target_s: float) -> int:
    """Points per (N, direction) so that one pass over the sweep takes about
    target_s seconds (grown until the probe itself is long enough to time)."""
    probe = 1 << 14
    limit = min(TOTAL, flat.size)
    while True:
        dt = oracle_sweep_once(flat, probe, nthreads)
        if dt >= min(1.0, target_s / 4) or probe >= limit:
            break
        probe = min(limit, probe * 4)
    pts = int(probe * target_s / max(dt, 1e-6))
    return max(1 << 12, min(limit, 1 << int(math.log2(max(pts, 1)))))


def cpu_baseline(flat, target_s: float = 12.0):
    cores = os.cpu_count() or 1
    pts = calibrate_oracle(flat, cores, target_s)
    dt = oracle_sweep_once(flat, pts, cores)
    nbytes = 16.0 * pts * len(SWEEP) * 2
    # the paper's own setting is one thread: the same oracle on one core, on a smaller sample
    pts1 = calibrate_oracle(flat, 1, 3.0)
    dt1 = oracle_sweep_once(flat, pts1, 1)
    single = {"value": 16.0 * pts1 * len(SWEEP) * 2 / dt1 / 1e9, "unit": UNIT, "cores": 1,
              "sample": f"{pts1} points per (N, direction), 1 thread, {dt1:.1f} s"}
    return {"value": nbytes / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"FP64 recursive radix-2 oracle, {pts} points per (N, direction) of the sweep "
                       f"({len(SWEEP)} sizes x 2 directions), {cores} threads over rows, {dt:.1f} s"),
            "single_core": single}


def run_reference(args):
    world, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2207_06803_gb300 import synth
    seed = synth.DEFAULT_SEED if args.seed is None else args.seed
    cores = os.cpu_count() or 1
    # One step = the oracle over a bounded sample of the sweep, sized so that
    # warmup + steps end within a few minutes.
    budget_s = 150.0 / max(1, args.steps + args.warmup)
    flat = synth.uniform_flat(seed, 0, 1 << 22)
    pts = min(calibrate_oracle(flat, cores, budget_s), 1 << 22)
    for _ in range(args.warmup):
        oracle_sweep_once(flat, pts, cores)
    times = [oracle_sweep_once(flat, pts, cores) for _ in range(args.steps)]
    total = sum(times)
    nbytes = 16.0 * pts * len(SWEEP) * 2
    value = nbytes * args.steps / total / 1e9
    sample = (f"FP64 recursive radix-2 oracle, {pts} points per (N, direction) of the sweep per step, "
              f"{cores} threads over rows")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_block(seed),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def config_block(seed):
    return {"workload": WORKLOAD, "sizes": SWEEP, "directions": ["forward", "inverse"],
            "elements_per_call": TOTAL, "algorithmic_bytes_per_call": BYTES_PER_CALL,
            "calls_per_step": 2 * len(SWEEP), "seed": seed, "layout": "contiguous rows, out of place",
            "l2": "inputs larger than L2 (512 MiB per call vs 129 MB L2); no flush"}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def run_gpu(args):
    import numpy as np
    import torch

    from paper_2207_06803_gb300 import gbfft, synth

    world, rank, local = dist_setup()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for the gbfft arm")
    torch.cuda.set_device(local)
    gbfft.lib()
    seed = synth.DEFAULT_SEED if args.seed is None else args.seed
    flat = synth.uniform_flat(seed, 0, TOTAL)
    d_in = torch.from_numpy(flat.view(np.float32)).to("cuda")
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.Stream()

    plans = []
    for n in SWEEP:
        for direction in (gbfft.GBFFT_FORWARD, gbfft.GBFFT_INVERSE):
            plans.append(((n, direction), gbfft.Plan(n, TOTAL // n, direction, args.dtype, variant=args.variant)))
    calls = len(plans)

    def step(events=None):
        for i, (_, p) in enumerate(plans):
            if events is not None:
                events[i][0].record(stream)
            p.execute(d_in, d_out, stream)
            if events is not None:
                events[i][1].record(stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    dev_index = local
    clocks = ClockSampler(dev_index)
    clocks.start()
    time.sleep(0.3)
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for _ in range(calls)]
          for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    t_start.record(stream)
    for s in range(args.steps):
        step(ev[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    max_ms = max_over_ranks(world, elapsed_ms)

    per_call_ms = [statistics.mean(ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(args.steps))
                   for i in range(calls)]
    per_size = {}
    for i, ((n, direction), _) in enumerate(plans):
        d = per_size.setdefault(str(n), {})
        d["fwd_gbs" if direction < 0 else "inv_gbs"] = BYTES_PER_CALL / (per_call_ms[i] * 1e-3) / 1e9
    dom = max(range(calls), key=lambda i: per_call_ms[i])
    (dom_n, dom_dir), dom_plan = plans[dom]
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    achieved = BYTES_PER_CALL / (per_call_ms[dom] * 1e-3) / 1e9
    info = dom_plan.info()
    kernel_key = f"stockham_rows_n{dom_n}_{'fwd' if dom_dir < 0 else 'inv'}_v{info['variant']}"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(kernel_key), "kernel": kernel_key,
                "radices": info["radices"], "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_src == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": BYTES_PER_CALL}

    # Accuracy of what was timed, after the timed region: every plan runs once more on the same
    # input and 256 seeded rows of its output are checked against the FP64 oracle.
    oracle_acc = {}
    if rank == 0:
        for (n, direction), p in plans:
            batch = TOTAL // n
            with torch.cuda.stream(stream):
                p.execute(d_in, d_out, stream)
            stream.synchronize()
            rows = synth.sample_rows(seed + n, batch, 256)
            y = sampled_rows(torch, np, d_out, batch, n, rows)
            x = flat[: batch * n].reshape(batch, n)[rows]  # (--sizes may name lengths that do not divide TOTAL)
            oracle_acc.setdefault(str(n), {})["fwd" if direction < 0 else "inv"] = \
                accuracy_vs_oracle(y, x, direction, gate(n, FP32_GATE))

    # Round trip as well: ||inv(fwd(x)) - N x|| / ||N x|| on 256 rows per size.
    roundtrip = {}
    with torch.cuda.stream(stream):
        for n in SWEEP:
            rows = 256
            xs = d_in[: 2 * n * rows]
            a = torch.empty_like(xs)
            b = torch.empty_like(xs)
            with gbfft.Plan(n, rows, gbfft.GBFFT_FORWARD) as pf, gbfft.Plan(n, rows, gbfft.GBFFT_INVERSE) as pi:
                pf.execute(xs, a, stream)
                pi.execute(a, b, stream)
                stream.synchronize()
            xr = xs.view(rows, n, 2).double()
            br = b.view(rows, n, 2).double()
            err = torch.linalg.vector_norm((br - n * xr).reshape(rows, -1), dim=1) / \
                torch.linalg.vector_norm((n * xr).reshape(rows, -1), dim=1)
            roundtrip[str(n)] = float(err.max().item())

    # End to end through the public host-buffer entry point: pinned host input
    # and output; H2D + transform + D2H of every call inside the timed region.
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(2, min(args.steps, 5))
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, np, flat, plans, stream, world, e2e_steps, calls)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(flat)

    others = None
    if rank == 0 and world == 1 and not args.no_other_configs:
        others = other_configs(args)

    value = world * args.steps * calls * BYTES_PER_CALL / (max_ms * 1e-3) / 1e9
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config_block(seed), parallelism="replicas" if world > 1 else "single GPU"),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * calls,
            "clocks": clk,
            "per_size_gbs": per_size,
            "frac_of_hbm_per_size": {k: {kk: vv / peak for kk, vv in v.items()} for k, v in per_size.items()},
            "oracle_rel_l2": oracle_acc,
            "oracle_all_pass": all(v["pass"] for d in oracle_acc.values() for v in d.values()),
            "roundtrip_rel_l2_max": roundtrip,
            "gpu": torch.cuda.get_device_name(),
            "other_configs": others,
        }
        print(json.dumps(line), flush=True)
    for _, p in plans:
        p.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def other_configs(args):
    """Short live runs of the other hot-path rows, summarised (errors recorded, never fatal)."""
    out = {}
    small = argparse.Namespace(**vars(args))
    small.steps = 40
    for name, fn in (("pr1", run_pr1), ("twopass", run_twopass), ("tc", lambda a: run_tc(a, dists=("uniform",))),
                     ("ragged", run_ragged), ("f64", run_f64), ("nd", run_nd),
                     ("serving", lambda a: run_serving(a, rates=(1000, 10000, 50000), scale=0.2, serial_rates=(1000,),
                                              per_length_rates=(10000,)))):
        try:
            r = fn(small)
        except Exception as e:  # a failing secondary measurement must not lose the headline line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
            continue
        if name == "twopass":
            out[name] = {n: {"two_pass_gbs": round(v["alg_gbs"], 1), "oracle_rel_l2_max": v["oracle"]["rel_l2_max"],
                             **({"cluster_gbs": round(v["cluster_gbs"], 1),
                                 "cluster_oracle_rel_l2_max": v["cluster_oracle"]["rel_l2_max"]}
                                if "cluster_gbs" in v else {})}
                         for n, v in r["per_size"].items()}
        elif name == "tc":
            out[name] = {k: {"gbs": round(v["gbs"], 1), "vs_fp32": round(v["vs_fp32"], 3),
                             "oracle_rel_l2_max": v["oracle"]["rel_l2_max"], "gate": v["oracle"]["gate"],
                             "roundtrip_rel_l2_max": v["roundtrip_rel_l2_max"]} for k, v in r["results"].items()}
        elif name == "nd":
            out[name] = {k: {"alg_gbs": round(v["alg_gbs"], 1), "frac_actual_of_hbm": round(v["frac_actual_of_hbm"], 3),
                             "oracle_rel_l2_max": v["oracle"]["rel_l2_max"]}
                         for k, v in r["per_shape"].items()}
        elif name == "f64":
            out[name] = {n: {"fwd_gflops": round(v["fwd"]["gflops"], 1), "fwd_gbs": round(v["fwd"]["gbs"], 1),
                             "oracle_rel_l2_max": v["oracle"]["rel_l2_max"],
                             "roundtrip_rel_l2_max": v["roundtrip_rel_l2_max"]} for n, v in r["per_size"].items()}
        elif name == "ragged":
            res = r["results"]
            out[name] = {k: res[k] for k in ("ragged_graph_tuned_us", "ragged_gbs", "per_size_us", "per_transform_us",
                                             "speedup_vs_per_size", "speedup_vs_per_transform", "items")}
            out[name]["oracle_rel_l2_max"] = res["oracle"]["rel_l2_max"]
        elif name == "pr1":
            out[name] = {k: r[k] for k in ("us", "gbs", "oracle", "cpu_naive_1core_s", "cpu_naive_all_cores_s")}
        else:
            out[name] = {"batching": {rate: {k: v[k] for k in ("p50_s", "p99_s", "req_per_s", "gb_per_s",
                                                               "service_over_10ms", "over_10ms_by_phase", "groups")}
                                      for rate, v in r["batching"].items()},
                         "per_length_groups": {rate: {k: v[k] for k in ("p50_s", "p99_s", "req_per_s", "groups")}
                                               for rate, v in r["per_length_groups"].items()},
                         "serial_queue": {rate: {k: v[k] for k in ("p50_s", "p99_s", "req_per_s")}
                                          for rate, v in r["serial_queue"].items()}}
    return out


def run_e2e(torch, np, flat, plans, stream, world, e2e_steps, calls):
    """End to end through gbfft_execute_host: pinned host input and output;
    H2D + transform + D2H of every call inside the timed region."""
    h_in = torch.from_numpy(flat.view(np.float32)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    with torch.cuda.stream(stream):
        for (_, p) in plans[:2]:
            p.execute_host(h_in, h_out, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(e2e_steps):
        for (_, p) in plans:
            p.execute_host(h_in, h_out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = max_over_ranks(world, e0.elapsed_time(e1))
    e2e_value = world * e2e_steps * calls * BYTES_PER_CALL / (e2e_ms * 1e-3) / 1e9
    return {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
            "h2d_bytes_per_step": calls * BYTES_PER_CALL // 2,
            "d2h_bytes_per_step": calls * BYTES_PER_CALL // 2,
            "path": "gbfft_execute_host on pinned host buffers (the kernels read and write them directly over NVLink-C2C)"}


# --------------------------------------------------------------------------
# Other configurations (one JSON line each; not the headline line)
# --------------------------------------------------------------------------

# --------------------------------------------------------------------------
# Accuracy of timed outputs against the FP64 oracle (always outside the timed
# regions: the outputs are copied back after timing, sampled rows only)
# --------------------------------------------------------------------------

FP32_GATE, TC_GATE, F64_GATE = 2e-7, 1e-6, 1e-15  # rel-L2 per log2(N)


def gate(n: int, per_log2: float) -> float:
    return per_log2 * max(1.0, math.log2(n))


def accuracy_vs_oracle(y, x, sign: int, tol: float, naive: bool = False) -> dict:
    """Per-row relative L2 error ||y - ref|| / ||ref|| of rows `y` (the device
    output, complex) against the FP64 oracle on the same input rows `x`, with
    max / mean / p99, the paper's form max|y - ref| / N (Sec. VI) and the gate."""
    import numpy as np

    import oracle
    x = np.ascontiguousarray(x, dtype=np.complex128)
    fn = oracle.dft_naive if naive else oracle.dft
    ref = fn(x, sign, nthreads=os.cpu_count() or 1)
    y = np.asarray(y, dtype=np.complex128).reshape(ref.shape)
    num = np.linalg.norm(y - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    err = np.where(den > 0, num / np.where(den > 0, den, 1.0), num)
    return {"rows": int(err.size), "rel_l2_max": float(err.max()), "rel_l2_mean": float(err.mean()),
            "rel_l2_p99": float(np.percentile(err, 99)), "max_abs_over_n": float(np.abs(y - ref).max() / x.shape[1]),
            "gate": tol, "pass": bool(err.max() <= tol)}


def sampled_rows(torch, np, d_out, batch: int, n: int, rows, complex_dtype=None):
    """Rows `rows` of a (batch, n) complex buffer on the device, copied to the host."""
    complex_dtype = complex_dtype or np.complex64
    floats_per_row = 2 * n
    idx = torch.from_numpy(np.asarray(rows, dtype=np.int64)).to(d_out.device)
    sel = d_out[: batch * floats_per_row].view(batch, floats_per_row).index_select(0, idx)
    return sel.cpu().numpy().view(complex_dtype)


def _time_ms(torch, fn, reps, stream):
    """Median CUDA-event time of fn() over reps runs on `stream` (after 3 warm-ups)."""
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _peak():
    peaks, src = measured_peaks()
    return float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)), src


def run_pr1(args):
    """The small reference case: forward c2c N = 64, batch 4096, complex64 rows uniform[-1, 1) from the
    default seed, every row checked against the oracle's direct DFT (the definition, Sec. II).  The
    2 MiB input stays in L2, so the GB/s (16 B per point) is not an HBM figure; the direct DFT on the
    host is timed on one core (the paper's single-thread setting) and on all cores."""
    import numpy as np
    import torch

    import oracle
    from paper_2207_06803_gb300 import gbfft, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n, batch = 64, 4096
    seed = synth.DEFAULT_SEED if args.seed is None else args.seed
    flat = synth.uniform_flat(seed, 0, n * batch)
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    d_out = torch.empty_like(d_in)
    with gbfft.Plan(n, batch, -1) as p:
        ms = _time_ms(torch, lambda: p.execute(d_in, d_out, stream), max(100, args.steps), stream)
        torch.cuda.synchronize()
        assert gbfft.gbfft_plan_device_status(p.handle) == 0
        info = p.info()
    y = d_out.cpu().numpy().view(np.complex64).reshape(batch, n)
    x = flat.reshape(batch, n)
    acc = accuracy_vs_oracle(y, x, -1, gate(n, FP32_GATE), naive=True)
    xd = x.astype(np.complex128)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.dft_naive(xd, -1, nthreads=1)
    t1 = time.perf_counter()
    oracle.dft_naive(xd, -1, nthreads=cores)
    t2 = time.perf_counter()
    return {"config": "pr1", "metric": "forward c2c N=64 batch=4096: time, GB/s (16 B/point) and error of every row "
                                       "against the FP64 direct DFT",
            "n": n, "batch": batch, "seed": seed, "radices": info["radices"], "us": 1e3 * ms,
            "gbs": 16.0 * n * batch / (ms * 1e-3) / 1e9, "l2_resident": True, "oracle": acc,
            "cpu_naive_1core_s": t1 - t0, "cpu_naive_all_cores_s": t2 - t1, "cpu_cores": cores}


def run_mixed(args):
    """Single-pass mixed-radix lengths p * 2^k (p = 3, 5, 7) from 10 to 3584, forward, about 2^26 points per
    call: GB/s (16 B/point) of the default plan and of every compiled variant of the length, and the default
    plan's error on 256 sampled rows against the FP64 oracle."""
    import numpy as np
    import torch
    from paper_2207_06803_gb300 import gbfft, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    peak, src = _peak()
    flat = synth.uniform_flat(synth.DEFAULT_SEED, 0, TOTAL)
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    d_out = torch.empty_like(d_in)
    sizes = [int(v) for v in args.sizes.split(",")] if args.sizes else \
        [n for n in synth.size_family(10, 4096) if n & (n - 1)]
    rows = {}
    for n in sizes:
        batch = TOTAL // n
        res = {"batch": batch, "variants": {}}
        with gbfft.Plan(n, batch, -1) as p:
            info = p.info()
            ms = _time_ms(torch, lambda: p.execute(d_in, d_out, stream), max(5, args.steps // 20), stream)
        gbs = 16.0 * n * batch / (ms * 1e-3) / 1e9
        r_chk = synth.sample_rows(synth.DEFAULT_SEED + n, batch, 256)
        res.update({"default_variant": info["variant"], "radices": info["radices"], "gbs": gbs,
                    "frac_of_hbm": gbs / peak,
                    "oracle": accuracy_vs_oracle(sampled_rows(torch, np, d_out, batch, n, r_chk),
                                                 flat[: batch * n].reshape(batch, n)[r_chk], -1, gate(n, FP32_GATE))})
        for v in range(gbfft.gbfft_num_variants(n)):
            with gbfft.Plan(n, batch, -1, variant=v) as p:
                msv = _time_ms(torch, lambda: p.execute(d_in, d_out, stream), max(5, args.steps // 40), stream)
            vi = gbfft.gbfft_variant_info(n, v)
            res["variants"][str(v)] = {"radices": vi["radices"], "rows_per_cta": vi["rows_per_cta"],
                                       "threads": vi["threads_per_cta"], "kind": gbfft.gbfft_variant_kind(n, v),
                                       "gbs": 16.0 * n * batch / (msv * 1e-3) / 1e9}
        rows[str(n)] = res
    return {"config": "mixed", "metric": "single-pass mixed-radix c2c GB/s (16 B/point) and oracle error",
            "unit": "GB/s", "points_per_call": TOTAL, "peak_gbs": peak, "peak_source": src, "per_size": rows}


def run_twopass(args):
    """Eq. 2 two-pass lengths 5120..16384 at 2^26 points per call."""
    import numpy as np
    import torch
    from paper_2207_06803_gb300 import gbfft, synth
    torch.cuda.set_device(0)
    flat = synth.uniform_flat(synth.DEFAULT_SEED, 0, TOTAL)
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream()
    peak, src = _peak()
    rows = {}
    for n in (5120, 6144, 7168, 8192, 10240, 12288, 14336, 16384, 20480, 24576, 28672, 32768, 65536):
        batch = TOTAL // n
        res = {}
        rows_chk = synth.sample_rows(synth.DEFAULT_SEED + n, batch, 64)
        x_chk = flat.reshape(-1)[: batch * n].reshape(batch, n)[rows_chk]
        with gbfft.Plan(n, batch, -1, k_outer=0) as p:  # Eq. 2 as two passes (two HBM round trips): the default
            info = p.info()
            ms = _time_ms(torch, lambda: p.execute(d_in, d_out, stream), max(5, args.steps // 20), stream)
        res["oracle"] = accuracy_vs_oracle(sampled_rows(torch, np, d_out, batch, n, rows_chk), x_chk, -1,
                                           gate(n, FP32_GATE))
        alg = 16.0 * n * batch / (ms * 1e-3) / 1e9
        res.update({"k_outer": info["k_outer"], "m_inner": info["m_inner"], "ms": ms, "alg_gbs": alg,
                    "actual_gbs_two_round_trips": 2 * alg, "frac_actual_of_hbm": 2 * alg / peak})
        if gbfft.gbfft_num_variants(n) > 0:  # one pass on a thread-block cluster (variant 0)
            with gbfft.Plan(n, batch, -1, variant=0) as p:
                rad = p.info()["radices"]
                ms1 = _time_ms(torch, lambda: p.execute(d_in, d_out, stream), max(5, args.steps // 20), stream)
            res["cluster_oracle"] = accuracy_vs_oracle(sampled_rows(torch, np, d_out, batch, n, rows_chk), x_chk, -1,
                                                       gate(n, FP32_GATE))
            alg1 = 16.0 * n * batch / (ms1 * 1e-3) / 1e9
            res.update({"cluster_radices": rad, "cluster_ms": ms1, "cluster_gbs": alg1,
                        "cluster_frac_of_hbm": alg1 / peak, "cluster_vs_two_pass": ms / ms1})
        rows[str(n)] = res
    return {"config": "twopass", "metric": "N > 4096: one pass on a thread-block cluster and Eq. 2 as two passes, "
                                           "c2c GB/s (16 B/point algorithmic)",
            "unit": "GB/s", "points_per_call": TOTAL, "peak_gbs": peak, "peak_source": src, "per_size": rows}


def run_nd(args):
    """Multi-dimensional transforms (last axis by the row kernel, the others by the column kernel, in
    place): 2-D and 3-D shapes at 2^26 points per call; GB/s on 16 B/point (algorithmic) and on the
    HBM traffic of one read and one write per axis pass."""
    import numpy as np
    import torch
    from paper_2207_06803_gb300 import gbfft, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    peak, src = _peak()
    flat = synth.uniform_flat(synth.DEFAULT_SEED, 0, TOTAL)
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    d_out = torch.empty_like(d_in)
    rows = {}
    for dims in ((64, 4096), (512, 1024), (128, 512), (64, 64, 256), (32, 128, 1024), (512, 8, 1024)):
        total = 1
        for v in dims:
            total *= v
        batch = TOTAL // total
        with gbfft.Plan(dims, batch, -1) as p:
            ms = _time_ms(torch, lambda: p.execute(d_in, d_out, stream), max(5, args.steps // 20), stream)
        alg = 16.0 * total * batch / (ms * 1e-3) / 1e9
        items = synth.sample_rows(synth.DEFAULT_SEED + total, batch, 4)
        y = sampled_rows(torch, np, d_out, batch, total, items)
        x = flat[: batch * total].reshape(batch, total)[items]
        import oracle
        ref = oracle.dft_nd(x.astype(np.complex128).reshape((-1,) + tuple(dims)), -1,
                            nthreads=os.cpu_count() or 1).reshape(len(items), total)
        err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        acc = {"items": int(len(items)), "rel_l2_max": float(err.max()), "rel_l2_mean": float(err.mean()),
               "max_abs_over_n": float(np.abs(y - ref).max() / total), "gate": gate(total, FP32_GATE),
               "pass": bool(err.max() <= gate(total, FP32_GATE))}
        rows["x".join(map(str, dims))] = {"batch": batch, "ms": ms, "alg_gbs": alg, "oracle": acc,
                                          "actual_gbs": alg * len(dims), "frac_actual_of_hbm": alg * len(dims) / peak}
    return {"config": "nd", "metric": "multi-dimensional c2c GB/s (16 B/point algorithmic; one HBM round trip per axis)",
            "unit": "GB/s", "points_per_call": TOTAL, "peak_gbs": peak, "peak_source": src, "per_shape": rows}


def run_pease(args):
    """Pease's constant-geometry factorisation (variant kind 5) against the default Stockham plan on
    the same lengths: N = 64, 256, 512, 4096 at 2^26 points per call, forward; GB/s on 16 B/point
    and the relative L2 error of 256 sampled rows against the FP64 oracle."""
    import numpy as np
    import torch
    from paper_2207_06803_gb300 import gbfft, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    peak, src = _peak()
    flat = synth.uniform_flat(synth.DEFAULT_SEED, 0, TOTAL)
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    d_out = torch.empty_like(d_in)
    rows = {}
    for n in (64, 256, 512, 4096):
        batch = TOTAL // n
        kinds = [gbfft.gbfft_variant_kind(n, v) for v in range(gbfft.gbfft_num_variants(n))]
        res = {}
        for name, variant in (("stockham_default", None), ("pease", kinds.index(5))):
            with gbfft.Plan(n, batch, -1, variant=variant) as p:
                ms = _time_ms(torch, lambda: p.execute(d_in, d_out, stream), max(5, args.steps // 20), stream)
                torch.cuda.synchronize()
            sample = synth.sample_rows(synth.DEFAULT_SEED + n, batch, 256)
            y = sampled_rows(torch, np, d_out, batch, n, sample)
            x = flat.reshape(batch, n)[sample]
            gbs = 16.0 * n * batch / (ms * 1e-3) / 1e9
            res[name] = {"ms": ms, "gbs": gbs, "frac_of_hbm": gbs / peak,
                         "oracle": accuracy_vs_oracle(y, x, -1, gate(n, FP32_GATE))}
        res["pease_vs_stockham"] = res["pease"]["gbs"] / res["stockham_default"]["gbs"]
        rows[str(n)] = res
    return {"config": "pease", "metric": "Pease constant-geometry vs Stockham c2c GB/s (16 B/point)",
            "unit": "GB/s", "points_per_call": TOTAL, "peak_gbs": peak, "peak_source": src, "per_size": rows}


FP64_NOMINAL_TFLOPS = 1.25  # GB300 dense FP64, nominal (no measured figure exists for it)


def run_f64(args):
    """Complex128 / FP64 path: N = 2^3..2^12 (and three mixed lengths), forward and inverse,
    2^26 points per call (1 GiB in, 1 GiB out); GB/s on 32 B/point, GFLOP/s on 5 N log2 N per
    transform against the nominal FP64 peak (this path is bound by the FP64 pipe, not HBM)."""
    import math
    import numpy as np
    import torch
    from paper_2207_06803_gb300 import gbfft, synth
    torch.cuda.set_device(0)
    total = TOTAL
    lo = synth.uniform_flat(synth.DEFAULT_SEED + 1, 0, total).astype(np.complex128)
    flat = synth.uniform_flat(synth.DEFAULT_SEED, 0, total).astype(np.complex128) + lo * 2.0 ** -26
    del lo
    d_in = torch.from_numpy(flat.view(np.float64)).cuda()
    d_out = torch.empty_like(d_in)
    d_rt = torch.empty_like(d_in)
    stream = torch.cuda.current_stream()
    rows = {}
    sizes = [int(v) for v in args.sizes.split(",")] if args.sizes else [1 << k for k in range(3, 13)] + [1536, 2560, 3584]
    for n in sizes:
        batch = total // n
        res = {}
        for direction, name in ((-1, "fwd"), (1, "inv")):
            with gbfft.Plan(n, batch, direction, dtype=gbfft.GBFFT_C2C_F64) as p:
                ms = _time_ms(torch, lambda: p.execute(d_in, d_out, stream), max(5, args.steps // 30), stream)
            flops = 5.0 * n * math.log2(n) * batch
            res[name] = {"ms": ms, "gbs": 32.0 * n * batch / (ms * 1e-3) / 1e9,
                         "gflops": flops / (ms * 1e-3) / 1e9,
                         "frac_of_fp64_nominal": flops / (ms * 1e-3) / (FP64_NOMINAL_TFLOPS * 1e12)}
        with gbfft.Plan(n, batch, -1, dtype=gbfft.GBFFT_C2C_F64) as pf, \
                gbfft.Plan(n, batch, 1, dtype=gbfft.GBFFT_C2C_F64) as pi:
            pf.execute(d_in, d_out, stream)
            pi.execute(d_out, d_rt, stream)
        torch.cuda.synchronize()
        rows_chk = synth.sample_rows(synth.DEFAULT_SEED + n, batch, 256)
        res["oracle"] = accuracy_vs_oracle(sampled_rows(torch, np, d_out, batch, n, rows_chk, np.complex128),
                                           flat[: batch * n].reshape(batch, n)[rows_chk], -1, gate(n, F64_GATE))
        sample = torch.from_numpy(synth.sample_rows(synth.DEFAULT_SEED, batch, 256)).cuda()
        a = d_rt[: 2 * n * batch].view(batch, 2 * n).index_select(0, sample).cpu().numpy().view(np.complex128)
        b = d_in[: 2 * n * batch].view(batch, 2 * n).index_select(0, sample).cpu().numpy().view(np.complex128) * n
        err = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
        res["roundtrip_rel_l2_max"] = float(err.max())
        rows[str(n)] = res
    return {"config": "f64", "metric": "complex128 FP64 c2c GFLOP/s (5 N log2 N) and GB/s (32 B/point)",
            "unit": "GFLOP/s", "points_per_call": total, "fp64_peak_tflops": FP64_NOMINAL_TFLOPS,
            "fp64_peak_source": "nominal GB300 dense FP64", "per_size": rows}


def run_tc(args, dists=("uniform", "gaussian_scaled")):
    """Tensor-core split precision vs the plain FP32 kernel: N=256 (2^18 rows), N=4096 (2^14 rows)."""
    import numpy as np
    import torch
    from paper_2207_06803_gb300 import gbfft, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    peak, src = _peak()
    out = {}
    stockham_sizes = [] if getattr(args, "sizes", None) else [256, 4096]
    for n, dist in [(n, d) for d in dists for n in stockham_sizes]:
        batch = TOTAL // n
        x = synth.uniform_flat(synth.DEFAULT_SEED, 0, TOTAL) if dist == "uniform" else \
            synth.gaussian_scaled_batch(synth.DEFAULT_SEED, n, batch).reshape(-1)
        d_in = torch.from_numpy(x.view(np.float32)).cuda()
        d_out = torch.empty_like(d_in)
        d_rt = torch.empty_like(d_in)
        for name, dt, var in (("fp32", 0, None), ("fp16x2", 1, 0), ("bf16x2", 2, 0), ("fp16x2_tcgen05", 1, 1),
                              ("bf16x2_tcgen05", 2, 1)):
            with gbfft.Plan(n, batch, -1, dt, variant=var) as pf, gbfft.Plan(n, batch, 1, dt, variant=var) as pi:
                ms = _time_ms(torch, lambda: pf.execute(d_in, d_out, stream), max(5, args.steps // 20), stream)
                pi.execute(d_out, d_rt, stream)
                torch.cuda.synchronize()
            xr = d_in.view(batch, 2 * n)[:4096].double()
            rr = d_rt.view(batch, 2 * n)[:4096].double()
            rt = (torch.linalg.vector_norm(rr - n * xr, dim=1) / torch.linalg.vector_norm(n * xr, dim=1)).max()
            gbs = BYTES_PER_CALL / (ms * 1e-3) / 1e9
            rows_chk = synth.sample_rows(synth.DEFAULT_SEED + n, batch, 256)
            acc = accuracy_vs_oracle(sampled_rows(torch, np, d_out, batch, n, rows_chk),
                                     x.reshape(batch, n)[rows_chk], -1, gate(n, FP32_GATE if dt == 0 else TC_GATE))
            out[f"{n}/{dist}/{name}"] = {"ms": ms, "gbs": gbs, "frac_of_hbm": gbs / peak, "oracle": acc,
                                         "roundtrip_rel_l2_max": float(rt)}
    # the direct DFT (one split-FP16 matrix product per 128 transforms) for small N
    direct_sizes = [int(v) for v in args.sizes.split(",")] if getattr(args, "sizes", None) else \
        [8, 16, 24, 32, 40, 48, 56, 64]
    for n, dist in [(n, d) for d in dists for n in direct_sizes]:
        batch = TOTAL // n
        x = synth.uniform_flat(synth.DEFAULT_SEED, 0, TOTAL) if dist == "uniform" else \
            synth.gaussian_scaled_batch(synth.DEFAULT_SEED, n, batch).reshape(-1)
        d_in = torch.from_numpy(x[: batch * n].view(np.float32)).cuda()
        d_out = torch.empty_like(d_in)
        d_rt = torch.empty_like(d_in)
        for name, dt, var in (("fp32", 0, None), ("fp16x2_direct", 1, 2), ("fp16x2_direct_tile_serial", 1, 3)):
            with gbfft.Plan(n, batch, -1, dt, variant=var) as pf, gbfft.Plan(n, batch, 1, dt, variant=var) as pi:
                ms = _time_ms(torch, lambda: pf.execute(d_in, d_out, stream), max(5, args.steps // 20), stream)
                pi.execute(d_out, d_rt, stream)
                torch.cuda.synchronize()
            xr = d_in.view(batch, 2 * n)[:4096].double()
            rr = d_rt.view(batch, 2 * n)[:4096].double()
            rt = (torch.linalg.vector_norm(rr - n * xr, dim=1) / torch.linalg.vector_norm(n * xr, dim=1)).max()
            gbs = 16.0 * n * batch / (ms * 1e-3) / 1e9
            rows_chk = synth.sample_rows(synth.DEFAULT_SEED + n, batch, 256)
            acc = accuracy_vs_oracle(sampled_rows(torch, np, d_out, batch, n, rows_chk),
                                     x[: batch * n].reshape(batch, n)[rows_chk], -1,
                                     gate(n, FP32_GATE if dt == 0 else TC_GATE))
            out[f"{n}/{dist}/{name}"] = {"ms": ms, "gbs": gbs, "frac_of_hbm": gbs / peak, "oracle": acc,
                                         "roundtrip_rel_l2_max": float(rt)}
    for key in list(out):
        n, dist, name = key.split("/")
        out[key]["vs_fp32"] = out[key]["gbs"] / out[f"{n}/{dist}/fp32"]["gbs"]
    return {"config": "tc", "metric": "tensor-core split-precision c2c GB/s vs plain FP32",
            "unit": "GB/s", "points_per_call": TOTAL, "peak_gbs": peak, "peak_source": src, "results": out}


def ragged_accuracy(torch, np, d_out, flat, sizes, offs, count):
    """Rel-L2 of `count` seeded transforms of a ragged output against the oracle, grouped by length."""
    from paper_2207_06803_gb300 import synth
    pick = synth.sample_rows(synth.DEFAULT_SEED + 11, sizes.size, count)
    y_all = d_out.cpu().numpy().view(np.complex64)
    errs, worst, passed, max_abs_n = [], {}, True, 0.0
    for n in sorted(set(sizes[pick].tolist())):
        sel = pick[sizes[pick] == n]
        idx = offs[sel][:, None] + np.arange(n)[None, :]
        a = accuracy_vs_oracle(y_all[idx], flat[idx], -1, gate(n, FP32_GATE))
        worst[str(n)] = a["rel_l2_max"]
        passed = passed and a["pass"]
        max_abs_n = max(max_abs_n, a["max_abs_over_n"])
        errs.append(a["rel_l2_max"])
    return {"transforms": int(pick.size), "rel_l2_max_per_size": worst, "rel_l2_max": float(max(errs)),
            "max_abs_over_n": max_abs_n, "gate": "2e-7 * log2(n) per size", "pass": passed}


def run_ragged(args):
    """10,000 transforms over the 41 lengths {2^k,3*2^k,5*2^k,7*2^k} in [8, 8192]: one persistent
    launch from a CUDA graph (autotuned tile shapes) vs one launch per length (grouped layout) vs one
    launch per transform."""
    import numpy as np
    import torch
    from paper_2207_06803_gb300 import gbfft, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sizes = synth.ragged_sizes(synth.DEFAULT_SEED, 10000)
    offs = synth.ragged_offsets(sizes)
    total = int(offs[-1] + sizes[-1])
    flat = synth.uniform_flat(synth.DEFAULT_SEED, 0, total)
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    d_out = torch.empty_like(d_in)
    nbytes = 16.0 * total
    reps = max(20, args.steps // 5)
    res = {"transforms": int(sizes.size), "distinct_sizes": int(len(set(sizes.tolist()))),
           "points": total, "algorithmic_bytes": nbytes}
    with gbfft.RaggedPlan(sizes, offs, -1) as rp:
        ms0 = _time_ms(torch, lambda: rp.execute(d_in, d_out, stream), reps, stream)
        # the same queue with every length on the run-time engine (schedules read from descriptors)
        gbfft.gbfft_ragged_set_engine(rp.handle, 0, 0)
        ms_rt = _time_ms(torch, lambda: rp.execute(d_in, d_out, stream), reps, stream)
        gbfft.gbfft_ragged_set_engine(rp.handle, 0, 1)
        res["ragged_graph_runtime_engine_us"] = 1e3 * ms_rt
        tuned = rp.autotune(d_in, d_out, reps=5)
        ms1 = _time_ms(torch, lambda: rp.execute(d_in, d_out, stream), reps, stream)
        res["ragged_graph_default_us"] = 1e3 * ms0
        res["ragged_graph_tuned_us"] = 1e3 * ms1
        res["oracle"] = ragged_accuracy(torch, np, d_out, flat, sizes, offs, 512)
        res["ragged_gbs"] = nbytes / (ms1 * 1e-3) / 1e9
        res["items"] = rp.num_items()
        res["engines"] = {str(n): gbfft.gbfft_ragged_engine(rp.handle, int(n)) for n in sorted(set(sizes.tolist()))}
        res["queue_order"] = gbfft.gbfft_ragged_queue_order(rp.handle)
        res["tile_splits"] = {str(n): gbfft.gbfft_ragged_tile_split(rp.handle, int(n))
                              for n in sorted(set(sizes.tolist()))}
        res["schedules"] = {str(n): gbfft.gbfft_ragged_schedule(rp.handle, int(n))
                            for n in sorted(set(sizes.tolist()))}
    if args.ragged_graph_only:
        return {"config": "ragged", "metric": "ragged batch GB/s on sum(16*N_i)", "unit": "GB/s", "results": res}
    # (i) one launch per distinct length over a grouped copy of the data
    order = np.argsort(sizes, kind="stable")
    grouped = np.concatenate([flat[offs[i]:offs[i] + sizes[i]] for i in order])
    g_in = torch.from_numpy(grouped.view(np.float32)).cuda()
    g_out = torch.empty_like(g_in)
    plans, start = [], 0
    for n in sorted(set(sizes.tolist())):
        cnt = int((sizes == n).sum())
        plans.append((gbfft.Plan(n, cnt, -1), 2 * start, 2 * (start + n * cnt)))
        start += n * cnt

    def per_size():
        for p, a, b in plans:
            p.execute(g_in[a:b], g_out[a:b], stream)
    ms2 = _time_ms(torch, per_size, reps, stream)
    res["per_size_launches"] = len(plans)
    res["per_size_us"] = 1e3 * ms2
    res["per_size_gbs"] = nbytes / (ms2 * 1e-3) / 1e9
    for p, _, _ in plans:
        p.close()
    # (ii) one launch per transform
    single = {n: gbfft.Plan(int(n), 1, -1) for n in set(sizes.tolist())}
    ptr_in, ptr_out = d_in.data_ptr(), d_out.data_ptr()
    calls = [(single[int(n)].handle, ptr_in + 8 * int(o), ptr_out + 8 * int(o)) for n, o in zip(sizes, offs)]
    sh = stream.cuda_stream

    def per_transform():
        for h, a, b in calls:
            gbfft.gbfft_execute(h, a, b, sh)
    ms3 = _time_ms(torch, per_transform, 5, stream)
    res["per_transform_launches"] = len(calls)
    res["per_transform_us"] = 1e3 * ms3
    res["per_transform_gbs"] = nbytes / (ms3 * 1e-3) / 1e9
    for p in single.values():
        p.close()
    res["speedup_vs_per_size"] = ms2 / ms1
    res["speedup_vs_per_transform"] = ms3 / ms1
    return {"config": "ragged", "metric": "ragged batch GB/s on sum(16*N_i)", "unit": "GB/s", "results": res}


def run_serving(args, rates=(1000, 2000, 5000, 10000, 20000, 50000), scale=1.0, serial_rates=(1000, 5000),
                per_length_rates=(10000, 50000)):
    """Open-loop Poisson arrivals; each request batch ~ U{1..256}, N uniform over
    {2^k,3*2^k,5*2^k,7*2^k} in [16, 16384]; 4 GiB budget; page-locked host buffers.  Continuous
    batching with one ragged launch per admission round and direction (lengths <= 8192) that reads
    and writes the host buffers directly, against the same with the rows copied through the device
    arena (staged), per-length groups and the serial queue.  Every group is timed by events (copies in, transform, copies out), so each request's
    latency splits into phases, and a request whose service exceeded 10 ms is attributed to its
    longest phase."""
    import numpy as np
    import torch
    from paper_2207_06803_gb300 import gbfft, synth
    torch.cuda.set_device(0)
    fam = np.asarray(synth.size_family(16, 16384))
    rng = np.random.Generator(np.random.Philox(key=synth.DEFAULT_SEED))
    templates = 128
    tn = fam[rng.integers(0, fam.size, size=templates)]
    tb = rng.integers(1, 257, size=templates)
    t_in, t_out = [], []
    for i in range(templates):
        x = synth.uniform_flat(synth.DEFAULT_SEED + i, 0, int(tn[i] * tb[i]))
        t_in.append(torch.from_numpy(x.view(np.float32)).pin_memory())
        t_out.append(torch.empty_like(t_in[-1]).pin_memory())
    budget = 4 << 30
    phase_names = ("host_s", "device_wait_s", "h2d_s", "kernel_s", "d2h_s", "observe_s")

    def drive(srv, rate, count, seed, timed):
        r = np.random.Generator(np.random.Philox(key=seed))
        pick = r.integers(0, templates, size=count)
        arr = np.cumsum(r.exponential(1.0 / rate, size=count))
        arr -= arr[0]
        srv.reset_stats()
        tickets = srv.replay([int(tn[k]) for k in pick], [int(tb[k]) for k in pick], [-1] * count,
                             [t_in[k] for k in pick], [t_out[k] for k in pick], arr)
        for t in tickets:
            srv.wait(t, 300.0)
        st = srv.stats()
        tm = np.array([srv.timing(t) for t in tickets])
        ph = [srv.phases(t) for t in tickets] if timed else None
        for t in tickets:
            srv.release(t)
        q, lat = tm[:, 0], tm[:, 1]
        service = lat - q
        st.update({"p999_s": float(np.percentile(lat, 99.9)), "queue_p99_s": float(np.percentile(q, 99)),
                   # requests whose service (admission to completion seen) took over 10 ms
                   "service_over_10ms": int((service > 0.01).sum()),
                   "max_service_s": float(service.max())})
        if timed:
            mat = np.array([[p[k] for k in phase_names] for p in ph])
            st["phase_p50_s"] = {k: float(np.percentile(mat[:, i], 50)) for i, k in enumerate(phase_names)}
            st["phase_p99_s"] = {k: float(np.percentile(mat[:, i], 99)) for i, k in enumerate(phase_names)}
            slow = np.where(service > 0.01)[0]
            st["over_10ms_by_phase"] = {}
            for j in slow:
                k = phase_names[int(np.argmax(mat[j]))]
                st["over_10ms_by_phase"][k] = st["over_10ms_by_phase"].get(k, 0) + 1
        return st

    def run_server(rates_, n_streams, warm_seed, count_of, **kw):
        out = {}
        timed = kw.get("phases", False)
        with gbfft.Server(mem_budget_bytes=budget, n_streams=n_streams, **kw) as srv:
            for n in fam.tolist():
                srv.prepare(int(n), -1)
            drive(srv, 5000, 1000, warm_seed, timed)  # warm-up
            for rate in rates_:
                count = count_of(rate)
                st = drive(srv, rate, count, rate, timed)
                out[str(rate)] = dict(st, requests=count, offered_req_per_s=rate)
        return out

    def count_full(rate):
        return max(500, int(scale * (20000 if rate >= 5000 else 10 * rate)))

    results = run_server(rates, 4, 7, count_full, phases=True)
    per_length = run_server(per_length_rates, 4, 9, count_full, phases=True, per_length=True)
    staged = run_server(per_length_rates, 4, 10, count_full, phases=True, staged=True)
    serial = run_server(serial_rates, 1, 8, lambda rate: max(500, int(scale * 3000)), serial=True)
    return {"config": "serving", "metric": "serving p50/p99 latency (s) and throughput",
            "budget_bytes": budget, "streams": 4, "request_templates": templates,
            "batching": results, "staged_copies": staged, "per_length_groups": per_length, "serial_queue": serial}


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config != "sweep":
        fn = {"pr1": run_pr1, "mixed": run_mixed, "twopass": run_twopass, "tc": run_tc, "ragged": run_ragged, "serving": run_serving, "pease": run_pease,
              "f64": run_f64, "nd": run_nd}[args.config]
        print(json.dumps(fn(args)), flush=True)
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
