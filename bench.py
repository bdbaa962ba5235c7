#!/usr/bin/env python3
"""Benchmark of the device-resident 19-point Jacobi sweep (one JSON line).

Default workload: the 129 x 129 x 257 grid, FP32 storage and arithmetic,
1000 sweeps kept on the device.  One step = the whole hot path over one
batch of synthetic inputs: copy-in (device-side rounding of the resident FP64
inputs into storage precision), 1000 sweeps, residual of the last sweep,
copy-out of the state.  ``value`` times that with inputs resident in HBM;
``e2e`` times the same through the C ABI from pinned host FP64 buffers, with
the host-device copies inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...    # the FP64 CPU oracle as the reference arm

Under torchrun each rank runs an independent replica on its own GPU (the
sweep of one grid is not sharded here); ``value`` is the sum over ranks of
point-updates divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "19-pt Jacobi Gpoint-updates/s"
UNIT = "Gpoint-updates/s"
BYTES_PER_POINT = {"f64": 112, "f32": 56, "bf16": 34}
DTYPE = {"f64": "f64", "f32": "f32", "bf16": "f32+bf16coef"}

WORKLOADS = {
    "config2": dict(I=129, J=129, K=257, sweeps=1000, prec="f32"),
    "config2-bf16": dict(I=129, J=129, K=257, sweeps=1000, prec="bf16"),
    "config2-f64": dict(I=129, J=129, K=257, sweeps=1000, prec="f64"),
    "config1": dict(I=33, J=33, K=65, sweeps=200, prec="f64"),
    "large": dict(I=513, J=513, K=1025, sweeps=100, prec="f32"),
    "large-bf16": dict(I=513, J=513, K=1025, sweeps=100, prec="bf16"),
}


def workload_name(w: dict) -> str:
    return f"{w['I']}x{w['J']}x{w['K']} {w['prec']} storage, {w['sweeps']} device-resident sweeps"


def n_interior(w: dict) -> int:
    return (w["I"] - 2) * (w["J"] - 2) * (w["K"] - 2)


def l2_note(w: dict) -> str:
    pitch = (w["I"] + 7) // 8 * 8
    ws = BYTES_PER_POINT[w["prec"]] * pitch * w["J"] * w["K"]
    return f"inputs larger than L2: {ws / 1e6:.0f} MB swept per sweep vs 129 MB L2; no flush"


# ---------------------------------------------------------------- helpers
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("jac_sweep.cu", "jac_common.cuh"):
        with open(os.path.join(ROOT, "paper_2002_12115_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(w: dict):
    """DRAM bytes per launch of the sweep kernel from a committed ncu summary,
    if it was taken on the current kernel source for this workload."""
    path = os.path.join(ROOT, "profiles", "k_sweep_traffic.md")
    if not os.path.exists(path):
        return None
    key = f"{w['I']}x{w['J']}x{w['K']} {w['prec']}"
    cur = kernel_source_hash()
    with open(path) as fh:
        for line in fh:
            m = re.match(r"\|\s*([^|]+?)\s*\|\s*([0-9a-f]{16})\s*\|\s*([0-9.eE+]+)\s*\|", line)
            if m and m.group(1) == key and m.group(2) == cur:
                return float(m.group(3))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not getattr(self, "out", ""):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- oracle arm
def oracle_sample(w: dict, min_seconds: float = 10.0, max_sweeps: int = 4000, chunk: int = 10):
    """The FP64 CPU oracle, as it stands, on the workload's grid: sweeps in
    chunks until about min_seconds of CPU time; returns Gpt/s and details."""
    import jacobi_inputs as ji
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    f = ji.himeno_fields(w["I"], w["J"], w["K"])
    p = f["p"]
    done, t_total = 0, 0.0
    while t_total < min_seconds and done < max_sweeps:
        t0 = time.perf_counter()
        p, _ = oracle.run(f, chunk, 0.8, p0=p)
        t_total += time.perf_counter() - t0
        done += chunk
    gpts = n_interior(w) * done / t_total / 1e9
    sample = (f"{done} FP64 oracle sweeps of the {w['I']}x{w['J']}x{w['K']} grid "
              f"({t_total:.1f} s on {cores} threads)")
    return gpts, cores, sample


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(2, min(w["sweeps"], 10))
    import jacobi_inputs as ji
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    f = ji.himeno_fields(w["I"], w["J"], w["K"])
    for _ in range(args.warmup):
        oracle.run(f, per_step, 0.8)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(f, per_step, 0.8)
    dt = time.perf_counter() - t0
    v = n_interior(w) * per_step * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(w) + f" (each step a bounded sample: {per_step} sweeps)",
                   "grid": [w["I"], w["J"], w["K"]], "sweeps_per_step": per_step},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} FP64 oracle sweeps per step on the workload grid"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- native arm
def run_native(args, w):
    import numpy as np
    import torch

    import jacobi_inputs as ji
    from paper_2002_12115_gb300 import Jacobi, lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib()  # fail loudly if the CUDA library is missing

    I, J, K, n, prec = w["I"], w["J"], w["K"], w["sweeps"], w["prec"]
    fields = ji.himeno_fields(I, J, K)
    names = list(fields)
    dev_fields = {k: torch.from_numpy(v).cuda() for k, v in fields.items()}
    host_fields = {}
    for k, v in fields.items():
        t = torch.empty(v.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = v
        host_fields[k] = t.numpy()
    p_host = torch.empty((K, J, I), dtype=torch.float64, pin_memory=True).numpy()
    p_dev = torch.empty((K, J, I), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    jac = Jacobi(I, J, K, prec, 0.8, stream)
    if args.tile_j or args.kdepth or args.tile_i:
        jac.set_plan(args.tile_j, args.kdepth, args.tile_i)

    sweep_ms = []

    def step(timed_sweeps: bool):
        jac.upload_tensors(dev_fields)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        jac.sweep(n)
        e1.record(stream)
        g = jac.residual()
        jac.download_tensor(p_dev)
        if timed_sweeps:
            sweep_ms.append((e0, e1))
        return g

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step(False)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            gosa = step(True)
        t1.record(stream)
        torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    if dist is not None:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    units = n_interior(w) * n * args.steps * world
    value = units / (ms * 1e-3) / 1e9
    launch_ms = sum(a.elapsed_time(b) for a, b in sweep_ms) / (n * args.steps)

    # end to end through the C ABI from pinned host buffers
    for _ in range(max(1, args.warmup // 2)):
        jac.upload(host_fields); jac.sweep(n); jac.residual(); jac.download(p_host)
    barrier()
    e_steps = max(1, args.steps)
    t0e = time.perf_counter()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(e_steps):
        jac.upload(host_fields)
        jac.sweep(n)
        jac.residual()
        jac.download(p_host)
    c1.record(stream)
    torch.cuda.synchronize()
    e_ms = max(c0.elapsed_time(c1), (time.perf_counter() - t0e) * 1e3)
    if dist is not None:
        tt = torch.tensor([e_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e_ms = float(tt.item())
    e2e = n_interior(w) * n * e_steps * world / (e_ms * 1e-3) / 1e9
    jac.close()

    # comparisons on the same GPU: the other precisions of the same grid
    variants = {}
    if not args.no_variants:
        for vp in ("f64", "bf16", "f32"):
            if vp == prec:
                continue
            with Jacobi(I, J, K, vp, 0.8, stream) as vj:
                vj.upload_tensors(dev_fields)
                vj.sweep(n); vj.residual()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                vj.sweep(n)
                b.record(stream)
                vj.residual()
                vms = a.elapsed_time(b)
                variants[vp] = {"value": n_interior(w) * n / (vms * 1e-3) / 1e9, "unit": UNIT,
                                "ms_per_sweep": vms / n,
                                "gbs": BYTES_PER_POINT[vp] * n_interior(w) / (vms / n * 1e-3) / 1e9}

    peak, peak_kind = measured_peak()
    bytes_launch = BYTES_PER_POINT[prec] * n_interior(w)
    achieved = bytes_launch / (launch_ms * 1e-3) / 1e9
    traffic = profiled_traffic(w)
    clocks = clk.summary()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        gpts, cores, sample = oracle_sample(w, min_seconds=args.cpu_seconds)
        cpu = {"value": gpts, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
            "config": {"workload": workload_name(w), "grid": [I, J, K], "sweeps": n, "prec": prec,
                       "omega": 0.8, "l2": l2_note(w),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "step": "device-side copy-in of resident FP64 inputs, sweeps, residual, copy-out"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic, "kernel": "k_sweep",
                         "algorithmic_bytes_per_launch": bytes_launch,
                         "launch_ms": launch_ms},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 13 * I * J * K * 8,
                    "d2h_bytes_per_step": I * J * K * 8 + 8},
            "gpu_launches": args.steps * (13 + n + 1),
            "clocks": clocks,
            "residual": gosa,
            "variants_same_gpu": variants,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="config2")
    ap.add_argument("--tile-j", type=int, default=0)
    ap.add_argument("--kdepth", type=int, default=0)
    ap.add_argument("--tile-i", type=int, default=0)
    ap.add_argument("--sweeps", type=int, default=0, help="override the workload's sweep count (profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.sweeps:
        w["sweeps"] = args.sweeps
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_native(args, w)


if __name__ == "__main__":
    main()
