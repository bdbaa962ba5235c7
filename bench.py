#!/usr/bin/env python3
"""Benchmark of the device-resident 19-point Jacobi sweep (one JSON line).

Default workload: the 513 x 513 x 1025 grid (about 270 M points), FP32
storage and arithmetic, 100 sweeps kept on the device.  One step = the whole
forward hot path over one batch of synthetic inputs: copy-in (device-side
rounding of the resident FP64 inputs into storage precision), 100 sweeps
(one persistent launch), residual of the last sweep, copy-out of the state.
``value`` times that with inputs resident in HBM; ``e2e`` times the same
through the C ABI from pinned host FP64 buffers, with the host-device copies
inside the timed region.  ``parity`` holds the result's error against the
FP64 CPU oracle run on the same inputs (the whole grid, all sweeps).

The line's ``compare`` block measures, on the same GPU: the BF16-coefficient
and FP64 paths of the same grid, the reverse pass of the last 20 of the 100
sweeps with a checkpoint every 5 (the rest of that workload), the 129 x 129 x
257 grid over 1000 sweeps in all three precisions, the per-sweep host-device
transfer variant of that grid, and the batched workload (512 grids of 17..129
points per side, 100 sweeps in one graph-replayed launch, against per-grid
launch loops).

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
# adjoint kernel: 14 arrays read, lambda written, FP64 dL/dwrk1 and dL/da3 read and written
ADJ_BYTES_PER_POINT = {"f64": 14 * 8 + 8 + 32, "f32": 14 * 4 + 4 + 32, "bf16": 11 * 2 + 3 * 4 + 4 + 32}
DTYPE = {"f64": "f64", "f32": "f32", "bf16": "f32+bf16coef"}

WORKLOADS = {
    "config2": dict(I=129, J=129, K=257, sweeps=1000, prec="f32"),
    "config2-bf16": dict(I=129, J=129, K=257, sweeps=1000, prec="bf16"),
    "config2-f64": dict(I=129, J=129, K=257, sweeps=1000, prec="f64"),
    "config1": dict(I=33, J=33, K=65, sweeps=200, prec="f64"),
    "large": dict(I=513, J=513, K=1025, sweeps=100, prec="f32"),
    "large-bf16": dict(I=513, J=513, K=1025, sweeps=100, prec="bf16"),
    "large-f64": dict(I=513, J=513, K=1025, sweeps=100, prec="f64"),
    "medium": dict(I=257, J=257, K=513, sweeps=100, prec="f32"),
    "profile": dict(I=257, J=257, K=257, sweeps=10, prec="f32"),
    # 3-D FFT block: the spectral step (inverse transform of U times the
    # heat-equation decay, energy sum) on a 512^3 complex grid
    "fft": dict(n=(512, 512, 512), prec="c32", alpha=1e-5),
    "fft-c64": dict(n=(512, 512, 512), prec="c64", alpha=1e-5),
    "fft-profile": dict(n=(256, 256, 256), prec="c32", alpha=1e-5),
    "fft-profile-c64": dict(n=(256, 256, 256), prec="c64", alpha=1e-5),
    "medium-bf16": dict(I=257, J=257, K=513, sweeps=100, prec="bf16"),
    "batch": dict(n_grids=512, sweeps=100, prec="f32"),
    "batch64": dict(n_grids=64, sweeps=100, prec="f32"),
    "batch-f64": dict(n_grids=512, sweeps=100, prec="f64"),
    "tuners": dict(n_grids=512, sweeps=100, prec="f32"),
    "oracle-configs": dict(),
    "sweep-latency": dict(I=33, J=33, K=65, sweeps=200, prec="f64"),
    "adjoint": dict(I=513, J=513, K=1025, sweeps=100, taped=20, C=5, prec="f32"),
    "adjoint-medium": dict(I=257, J=257, K=513, sweeps=40, taped=20, C=5, prec="f32"),
    "adjoint-65": dict(I=65, J=65, K=129, sweeps=50, taped=50, C=10, prec="f64"),
    "adjoint-f64": dict(I=513, J=513, K=1025, sweeps=100, taped=20, C=5, prec="f64"),
}


def n_interior(w: dict) -> int:
    return (w["I"] - 2) * (w["J"] - 2) * (w["K"] - 2)


def workload_name(w: dict) -> str:
    return f"{w['I']}x{w['J']}x{w['K']} {w['prec']} storage, {w['sweeps']} device-resident sweeps"


def l2_note(w: dict) -> str:
    pitch = (w["I"] + 7) // 8 * 8
    ws = BYTES_PER_POINT[w["prec"]] * pitch * w["J"] * w["K"]
    if ws > 129e6:
        return f"inputs larger than L2: {ws / 1e6:.0f} MB swept per sweep vs 129 MB L2; no flush"
    return (f"working set ({ws / 1e6:.0f} MB) fits in the 129 MB L2; no flush: the steady state of "
            "resident sweeps, whose inputs stay in L2 from sweep to sweep")


# ---------------------------------------------------------------- helpers
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 operations (DADD, DMUL, DFMA, each one issue of the FP64 pipe) per
# interior point of a non-residual FP64 sweep: 9 in the three b-brackets, 9
# fused terms of s0, one fused and one plain product for ss, one fused update.
F64_OPS_PER_POINT = 21
# GB300 issues two FP64 thread operations per SM per clock (the ncu peak of
# sm__sass_thread_inst_executed_op_dfma_pred_on is 2 per SM per cycle).
F64_OPS_PER_SM_CLK = 2
GB300_SMS = 152


def f64_alu_peak_gops():
    """FP64 ALU ceiling in G FP64 operations/s: 2 per SM per clock x 152 SMs x
    the maximum SM clock from MEASURED_PEAKS.json (2070 MHz if absent)."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz = float(json.load(fh).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return F64_OPS_PER_SM_CLK * GB300_SMS * mhz * 1e6 / 1e9


def variant_roofline(prec: str, gpts: float) -> dict:
    """Roofline of one sweep variant: HBM for FP32 and BF16 storage, the FP64
    ALU for FP64 (its 112 B per point would need more than the HBM peak only
    above 61 Gpoint-updates/s; the FP64 pipe caps it near 30)."""
    if prec == "f64":
        ach = F64_OPS_PER_POINT * gpts
        peak = f64_alu_peak_gops()
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "G FP64 op/s", "frac": ach / peak,
                "peak_kind": "derived: 2 FP64 ops per SM per clock x 152 SMs x max SM clock",
                "ops_per_point": F64_OPS_PER_POINT}
    peak, kind = measured_peak()
    ach = BYTES_PER_POINT[prec] * gpts
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_kind": kind}


SWEEP2_FILES = ("jac_sweep2.cu", "jac_sweep_kernel.cuh", "jac_common.cuh")


def sweep_split(w, prec, n, fuse=0):
    """(two-sweep passes, single sweeps) of a call of n sweeps under the
    library's plan for this grid (fuse 0: the library's choice): an even
    number of passes when the resolved plan takes them and n >= 4."""
    from paper_2002_12115_gb300.binding import resolve_plan
    f = resolve_plan(w["I"], w["J"], w["K"], prec, fuse=fuse)["fuse"]
    if prec != "f32" or f != 2 or n < 4:
        return 0, n
    n_pass = (n // 2) & ~1
    return n_pass, n - 2 * n_pass


def sweep_roofline(w, prec, n, ms, fuse=0) -> dict:
    """Roofline of one call of n sweeps that took ms: HBM (FP32, BF16) or the
    FP64 ALU for single sweeps; for two-sweep passes HBM at the pass's own
    algorithmic bytes (every array read once and the state written once per
    pass: 56 B per point per pass, 28 B per point-update), with the ceiling
    that single sweeps' 56 B per point-update put on the same bandwidth."""
    npts = n_interior(w)
    gpts = npts * n / (ms * 1e-3) / 1e9
    n_pass, rest = sweep_split(w, prec, n, fuse)
    peak, kind = measured_peak()
    key = f"{w['I']}x{w['J']}x{w['K']} {prec}"
    if n_pass == 0:
        r = variant_roofline(prec, gpts)
        r.update({"kernel": "k_sweep", "algorithmic_bytes_per_launch": BYTES_PER_POINT[prec] * npts * n})
        per_sweep = profiled_traffic(key)
        traffic = per_sweep * n if per_sweep else None
    else:
        bytes_launch = BYTES_PER_POINT[prec] * npts * (n_pass + rest)
        ach = bytes_launch / (ms * 1e-3) / 1e9
        ceiling = peak / BYTES_PER_POINT[prec]
        r = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_kind": kind,
             "kernel": "k_sweep2 (two sweeps per pass)" + (f" + {rest} single sweeps" if rest else ""),
             "passes_per_launch": n_pass, "algorithmic_bytes_per_launch": bytes_launch,
             "bytes_per_point_update": BYTES_PER_POINT[prec] / 2,
             "single_sweep_ceiling": {"gpts": ceiling, "value_over_ceiling": gpts / ceiling,
                                      "reading": "the rate single sweeps would reach at the full measured HBM "
                                                 "bandwidth (56 B per point-update)"},
             "reading": "a pass reads every array once per two point-updates; frac counts those bytes "
                        "(28 B per point-update) against the copy peak, and the pass is bound by latency, "
                        "not DRAM; the bandwidth fraction of single sweeps on the same grid (56 B per "
                        "point-update) is compare." + prec + "_single_sweeps"}
        per_pass = profiled_traffic(key + " two-sweep pass", SWEEP2_FILES)
        traffic = per_pass * n_pass if (per_pass and rest == 0) else None
    r["traffic"] = traffic
    if traffic:
        dram = traffic / (ms * 1e-3) / 1e9
        r.update({"dram_achieved": dram, "dram_frac": dram / peak})
    return r


def code_of(text: str) -> str:
    """A CUDA/C++ source without its comments and with its whitespace
    collapsed: what the compiler sees of it (the files have no string that
    holds a comment marker)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(names=("jac_sweep_kernel.cuh", "jac_common.cuh")) -> str:
    """First 16 hex digits of the sha256 of the kernel sources' code (comments
    and whitespace do not change it)."""
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2002_12115_gb300", "csrc", name)) as fh:
            h.update(code_of(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(key: str, kernel_files=("jac_sweep_kernel.cuh", "jac_common.cuh")):
    """DRAM bytes per unit (one sweep) of a kernel from the committed ncu
    summary, if it was taken on the current kernel source for this key."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash(kernel_files)
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
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
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


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest of x over all ranks (x itself on one process)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, ms: float, world: int, dist=None, device="cuda") -> tuple:
    """Whole-job throughput of independent replicas: the units of all ranks
    over the slowest rank's time.  Returns (value in units/s, max ms)."""
    ms_max = max_over_ranks(ms, dist, device)
    return units_per_rank * world / (ms_max * 1e-3), ms_max


def events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# --------------------------------------------------------------- oracle arm
def _sweeps_per_chunk(w: dict, target_s: float, gpts_guess: float) -> int:
    """Sweeps per timed oracle call so that one call takes about target_s."""
    return max(1, min(10, int(target_s * gpts_guess * 1e9 / n_interior(w))))


def oracle_sample(w: dict, min_seconds: float = 10.0, max_sweeps: int = 4000, fields=None):
    """The FP64 CPU oracle, as it stands, on the workload's grid: sweeps in
    chunks until about min_seconds of CPU time; returns Gpt/s and details.
    fields: the workload's inputs if the caller has them (else generated)."""
    import jacobi_inputs as ji
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    f = fields if fields is not None else ji.himeno_fields(w["I"], w["J"], w["K"])
    chunk = _sweeps_per_chunk(w, 1.0, 0.7)
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


def oracle_one_core(w: dict, seconds: float = 3.0, fields=None):
    """The same oracle on one thread, for a few seconds: Gpt/s."""
    import jacobi_inputs as ji
    import oracle
    cores = oracle.set_threads(0)
    oracle.set_threads(1)
    try:
        f = fields if fields is not None else ji.himeno_fields(w["I"], w["J"], w["K"])
        chunk = _sweeps_per_chunk(w, 1.0, 0.09)
        p = f["p"]
        done, t_total = 0, 0.0
        while t_total < seconds:
            t0 = time.perf_counter()
            p, _ = oracle.run(f, chunk, 0.8, p0=p)
            t_total += time.perf_counter() - t0
            done += chunk
    finally:
        oracle.set_threads(cores)
    return n_interior(w) * done / t_total / 1e9


TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 3e-3}


def oracle_parity(w: dict, fields: dict, p_gpu, gosa_gpu: float) -> dict:
    """The GPU result of the workload (state and residual after all its
    sweeps) against the FP64 CPU oracle run on the whole grid from the same
    inputs, rounded to the storage precision; for FP32-stored states the
    oracle rounds its state to FP32 after every sweep (the problem such a
    state solves).  Relative errors: max|dp| / max|p| and |dgosa| / gosa."""
    import numpy as np

    import oracle
    oracle.build()
    prec = w["prec"]
    fr = oracle.round_inputs(fields, prec)
    state = "f64" if prec == "f64" else "f32"
    t0 = time.perf_counter()
    wp, wg = oracle.run(fr, w["sweeps"], 0.8, state=state)
    dt = time.perf_counter() - t0
    del fr
    ep = float(np.abs(p_gpu - wp).max() / np.abs(wp).max())
    eg = abs(gosa_gpu - wg) / abs(wg)
    out = {"p_err": ep, "gosa_err": eg, "tol": TOL[prec], "pass": bool(ep <= TOL[prec] and eg <= TOL[prec]),
           "oracle_gosa": wg, "oracle_seconds": dt, "oracle_threads": oracle.set_threads(0),
           "sample": f"the whole grid, all {w['sweeps']} sweeps",
           "reference": ("FP64 CPU oracle on the same inputs" if prec == "f64" else
                         f"FP64 CPU oracle on the inputs rounded as {prec} storage rounds them, state rounded "
                         "to FP32 after every sweep")}
    if prec != "f64":
        out["reading"] = ("an FP32-stored state differs from the pure-FP64 iteration by its own rounding "
                          "(the residual by about 1e-4 relative on this grid, compare.residual_vs_f64_gpu); "
                          "the tolerance applies to the problem the stored precision solves")
    return out


def oracle_configs():
    """The FP64 CPU oracle, as it stands, on every workload configuration, on
    this host's cores: full runs where they take seconds, bounded samples
    (stated) elsewhere.  Input generation is outside the timed calls."""
    import jacobi_inputs as ji
    import oracle
    oracle.build()
    cores = oracle.set_threads(0)
    out = {}

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    def interior(I, J, K):
        return (I - 2) * (J - 2) * (K - 2)

    f = ji.himeno_fields(33, 33, 65)
    dt = timed(lambda: oracle.run(f, 200, 0.8))
    out["33x33x65 f64, 200 sweeps"] = {"seconds": dt, "gpts": interior(33, 33, 65) * 200 / dt / 1e9,
                                       "sample": "full run"}
    f = ji.himeno_fields(129, 129, 257)
    dt = timed(lambda: oracle.run(f, 1000, 0.8))
    out["129x129x257, 1000 sweeps"] = {"seconds": dt, "gpts": interior(129, 129, 257) * 1000 / dt / 1e9,
                                       "sample": "full run"}
    f = ji.himeno_fields(65, 65, 129)
    tg = ji.target_field(65, 65, 129)
    dt = timed(lambda: oracle.adjoint(f, 50, tg, 0.8))
    out["65x65x129 f64 adjoint, T = 50"] = {"seconds": dt, "sample": "full run: 50 sweeps forward (all states "
                                                                     "kept), 50 reverse-mode sweeps"}
    dims = ji.batch_dims(512)[:64]
    grids = [ji.himeno_fields(I, J, K, seed=42 + g) for g, (I, J, K) in enumerate(dims)]
    dt = timed(lambda: [oracle.run(fg, 100, 0.8) for fg in grids])
    pts = sum(interior(*d) for d in dims)
    out["512 grids, 100 sweeps"] = {"seconds_sample": dt, "gpts": pts * 100 / dt / 1e9,
                                    "sample": f"the first 64 of the 512 grids ({pts} interior points of "
                                              "126,983,056), all 100 sweeps each"}
    del grids
    f = ji.himeno_fields(513, 513, 65)
    dt = timed(lambda: oracle.run(f, 3, 0.8))
    g = interior(513, 513, 65) * 3 / dt / 1e9
    out["513x513x1025, 100 sweeps"] = {"gpts": g, "seconds_extrapolated": interior(513, 513, 1025) * 100 / g / 1e9,
                                       "sample": "3 sweeps of a 513x513x65 slab (same i-j plane), extrapolated "
                                                 "by interior point-updates"}
    return {"metric": METRIC + " (FP64 CPU oracle, every configuration)", "unit": UNIT, "cores": cores,
            "kind": "oracle", "configs": out}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if "I" not in w:
        w = WORKLOADS["config2"]
    # each step a bounded sample of the workload: about 0.7 s of oracle sweeps
    per_step = min(w["sweeps"], _sweeps_per_chunk(w, 0.7, 0.7))
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
def device_fields(I, J, K, seed=42):
    import jacobi_inputs as ji
    return ji.himeno_fields_torch(I, J, K, seed=seed, device="cuda")


def bench_single(args, w, stream):
    """Steps of one grid: device-side copy-in, n sweeps, residual, copy-out."""
    import torch

    from paper_2002_12115_gb300 import Jacobi
    I, J, K, n, prec = w["I"], w["J"], w["K"], w["sweeps"], w["prec"]
    dev = device_fields(I, J, K)
    host = None
    if args.need_host:
        # host copies of the same inputs (bitwise those of the numpy
        # generator), for the end-to-end steps and the oracle
        host = {k: v.cpu() for k, v in dev.items()}
    p_dev = torch.empty((K, J, I), dtype=torch.float64, device="cuda")
    jac = Jacobi(I, J, K, prec, 0.8, stream)
    if args.tile_j or args.kdepth or args.tile_i or args.fuse:
        jac.set_plan(args.tile_j, args.kdepth, args.tile_i, args.fuse)
    sweep_ev = []

    def step(record):
        jac.upload_tensors(dev)
        e0, e1 = events()
        e0.record(stream)
        jac.sweep(n)
        e1.record(stream)
        g = jac.residual()
        jac.download_tensor(p_dev)
        if record:
            sweep_ev.append((e0, e1))
        return g

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if args.dist is not None:
        args.dist.barrier()
    t0, t1 = events()
    with ClockSampler(args.local) as clk:
        t0.record(stream)
        for _ in range(args.steps):
            gosa = step(True)
        t1.record(stream)
        torch.cuda.synchronize()
    return {"ms": t0.elapsed_time(t1), "launch_ms": statistics.mean(a.elapsed_time(b) for a, b in sweep_ev),
            "residual": gosa, "jac": jac, "dev": dev, "host": host, "p": p_dev, "clocks": clk.summary()}


def bench_e2e(args, w, jac, stream, want_residual, fields_t, f32_host=False):
    """The same step through the C ABI from pinned host buffers: every step
    copies its thirteen inputs in, sweeps, and copies the state and the
    residual out, all inside the timed region.  f32_host: the inputs as FP32
    host arrays (jac_upload_f32_async / jac_download_f32_async; the numbers
    an FP32-stored problem holds), else FP64.  Two contexts on two streams
    take the steps in turn: one step's host-to-device copies run on the copy
    engine while the previous step's sweeps hold the SMs, and the previous
    step's results are copied out while this step sweeps."""
    import numpy as np
    import torch

    import jacobi_inputs as ji
    from paper_2002_12115_gb300 import Jacobi
    I, J, K, n = w["I"], w["J"], w["K"], w["sweeps"]

    def pinned(shape):
        return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()

    if f32_host:
        # the inputs as FP32 numbers (what FP32 storage holds), in pinned memory
        host = {}
        for k, v in fields_t.items():
            t = torch.empty(v.shape, dtype=torch.float32, pin_memory=True)
            t.copy_(v.float())
            host[k] = t.numpy()
        p_host = [torch.empty((K, J, I), dtype=torch.float32, pin_memory=True).numpy() for _ in range(2)]
    else:
        host = {}
        for k, v in fields_t.items():                        # pinned FP64 inputs
            t = torch.empty(v.shape, dtype=torch.float64, pin_memory=True)
            t.copy_(v)
            host[k] = t.numpy()
        p_host = [pinned((K, J, I)) for _ in range(2)]
    res_host = [pinned((1,)) for _ in range(2)]
    stream2 = torch.cuda.Stream()
    jac2 = Jacobi(I, J, K, w["prec"], 0.8, stream2, async_upload=True)
    if args.tile_j or args.kdepth or args.tile_i or args.fuse:
        jac2.set_plan(args.tile_j, args.kdepth, args.tile_i, args.fuse)
    ctxs = (jac, jac2)
    residuals = []

    up = (lambda c: c.upload_f32_async(host)) if f32_host else (lambda c: c.upload_async(host))
    down = (lambda c, o, r: c.download_f32_async(o, r)) if f32_host else (lambda c, o, r: c.download_async(o, r))

    def run(steps):
        for k in range(steps):
            cur, prev = ctxs[k % 2], ctxs[(k - 1) % 2]
            up(cur)
            if k >= 1:                       # the previous step's results, behind its sweeps
                down(prev, p_host[(k - 1) % 2], res_host[(k - 1) % 2])
            cur.sweep(n)
            if k >= 1:
                prev.sync()
                residuals.append(float(res_host[(k - 1) % 2][0]))
        last = ctxs[(steps - 1) % 2]
        down(last, p_host[(steps - 1) % 2], res_host[(steps - 1) % 2])
        last.sync()
        residuals.append(float(res_host[(steps - 1) % 2][0]))

    run(max(2, args.warmup // 2))
    torch.cuda.synchronize()
    if args.dist is not None:
        args.dist.barrier()
    t0 = time.perf_counter()
    run(args.steps)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    jac2.close()
    # same inputs and a bitwise-reproducible sweep: every step's residual is
    # the same, and that of the device-resident run (for FP32 host arrays the
    # stored values are the same numbers, so bitwise too)
    if len(set(residuals)) != 1 or not abs(residuals[0] - want_residual) <= 1e-5 * abs(want_residual):
        raise RuntimeError(f"end-to-end residuals {sorted(set(residuals))} against the device-resident "
                           f"run's {want_residual}")
    del host, p_host
    return ms


def bench_unhoisted_grid(w, sweeps=20):
    """The per-sweep transfer variant on a grid of its own (host inputs)."""
    import jacobi_inputs as ji
    from paper_2002_12115_gb300 import Jacobi
    host = ji.himeno_fields(w["I"], w["J"], w["K"])
    with Jacobi(w["I"], w["J"], w["K"], w["prec"], 0.8) as jac:
        v = bench_unhoisted(w, jac, host, sweeps)
    return {"value": v, "unit": UNIT, "grid": [w["I"], w["J"], w["K"]], "prec": w["prec"],
            "what": "every sweep copies the 13 host FP64 arrays in and p out (jac_sweep_unhoisted)"}


def bench_unhoisted(w, jac, host, sweeps=20):
    """Per-sweep copy-in / copy-out (what hoisting avoids), same grid."""
    import numpy as np
    import torch
    jac.sweep_unhoisted(2, host, np.array(host["p"]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    jac.sweep_unhoisted(sweeps, host, np.array(host["p"]))
    torch.cuda.synchronize()
    return n_interior(w) * sweeps / (time.perf_counter() - t0) / 1e9


def bench_variant(w, prec, dev, stream, sweeps, fuse=0):
    """Gpt/s of a precision on a grid (device-resident inputs); fuse as in
    the launch plan (0: the library's choice)."""
    from paper_2002_12115_gb300 import Jacobi
    with Jacobi(w["I"], w["J"], w["K"], prec, 0.8, stream) as vj:
        if fuse:
            vj.set_plan(0, 0, 0, fuse)
        vj.upload_tensors(dev)
        vj.sweep(max(2, sweeps // 10)); vj.residual()
        a, b = events()
        a.record(stream)
        vj.sweep(sweeps)
        b.record(stream)
        vj.residual()
        ms = a.elapsed_time(b)
    gbs = BYTES_PER_POINT[prec] * n_interior(w) / (ms / sweeps * 1e-3) / 1e9
    gpts = n_interior(w) * sweeps / (ms * 1e-3) / 1e9
    roofline = sweep_roofline(w, prec, sweeps, ms, fuse)
    return {"value": gpts, "unit": UNIT, "ms_per_sweep": ms / sweeps, "fuse": fuse,
            "gbs": gbs, "grid": [w["I"], w["J"], w["K"]], "prec": prec, "roofline": roofline}


def residual_vs_f64(w, dev, stream, sweeps):
    """The residual after `sweeps` sweeps of the workload's precision against
    the FP64 GPU run of the same grid from the same inputs (relative): the
    stored precision's own error on the observable the method reports.  This
    is the gap to the pure-FP64 problem, not the parity figure (that one is
    against the oracle on the rounded problem)."""
    from paper_2002_12115_gb300 import Jacobi
    res = {}
    prec = w["prec"]
    for vp in (prec, "f64"):
        with Jacobi(w["I"], w["J"], w["K"], vp, 0.8, stream) as vj:
            vj.upload_tensors(dev)
            vj.sweep(sweeps)
            res[vp] = vj.residual()
    return {"sweeps": sweeps, "gosa": res[prec], "gosa_f64": res["f64"],
            "rel_err": abs(res[prec] - res["f64"]) / abs(res["f64"]),
            "reading": "gap of the stored-precision iteration to the pure-FP64 one; no tolerance applies "
                       "(the FP32 bar is met against the rounded problem, see parity)"}


def bench_batch(args, stream, sweeps=100, steps=3, autotune=True, loops=True, tuner="cd", prec="f32",
                n_grids=512):
    """512 grids, dims drawn from {17, .., 129}: one graph-replayed persistent
    launch per step against loops of per-grid launches.  The plan search runs
    for FP32 storage; other precisions take the library's default plan.
    n_grids < 512: the first n_grids of the same draw (a profiling subset)."""
    import torch

    import jacobi_inputs as ji
    from paper_2002_12115_gb300 import JacobiBatch
    dims = ji.batch_dims(512)[:n_grids]
    npts = sum((I - 2) * (J - 2) * (K - 2) for I, J, K in dims)
    b = JacobiBatch(dims, prec, 0.8, stream)
    for g, (I, J, K) in enumerate(dims):
        b.upload_tensors(g, ji.himeno_fields_torch(I, J, K, seed=42 + g))
    plan = None
    if autotune and prec == "f32":
        from paper_2002_12115_gb300 import autotune as at
        if tuner == "ga":
            plan = at.ga_tune_batch(b, M=10, T=10, n_sweeps=10, reps=2)
        else:
            plan = at.tune_batch(b, n_sweeps=10, reps=2, passes=1)
    b.sweep(sweeps)          # capture + warm-up
    b.sweep(sweeps)
    a, e = events()
    a.record(stream)
    for _ in range(steps):
        b.sweep(sweeps)
    e.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / steps
    out = {"value": npts * sweeps / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
           "grids": len(dims), "points": npts, "sweeps": sweeps,
           "gbs": BYTES_PER_POINT[prec] * npts * sweeps / (ms * 1e-3) / 1e9,
           "launches_per_step": 1, "plan": plan, "info": b.info()}
    if loops:
        for key, per_sweep, launches in (("per_grid_launches", False, len(dims)),
                                         ("per_grid_per_sweep_launches", True, len(dims) * sweeps)):
            a, e = events()
            a.record(stream)
            b.sweep_loop(sweeps, per_sweep=per_sweep)
            e.record(stream)
            torch.cuda.synchronize()
            ms_l = a.elapsed_time(e)
            out[key] = {"value": npts * sweeps / (ms_l * 1e-3) / 1e9, "launches": launches}
    b.close()
    return out


def bench_tuners(stream, sweeps=100):
    """Launch-plan searches on the 512-grid batch, each from scratch: the
    default plan, coordinate descent (1 and 2 passes) and the paper's GA
    (M = T = 10, two seeds).  Reports each plan's rate, plans measured and the
    search time."""
    import torch

    import jacobi_inputs as ji
    from paper_2002_12115_gb300 import JacobiBatch
    from paper_2002_12115_gb300 import autotune as at
    dims = ji.batch_dims(512)
    npts = sum((I - 2) * (J - 2) * (K - 2) for I, J, K in dims)
    b = JacobiBatch(dims, "f32", 0.8, stream)
    for g, (I, J, K) in enumerate(dims):
        b.upload_tensors(g, ji.himeno_fields_torch(I, J, K, seed=42 + g))
    count = {"n": 0}
    set_plan = b.set_plan

    def counted(*a, **k):
        count["n"] += 1
        return set_plan(*a, **k)
    b.set_plan = counted

    def rate():
        b.sweep(sweeps, residuals=False)
        return npts * sweeps / at.time_call(lambda: b.sweep(sweeps, residuals=False), 3, stream) / 1e9

    set_plan(0, None, None)
    out = {"default": {"value": rate(), "plans_measured": 0}}
    runs = (("cd_1pass", lambda: at.tune_batch(b, n_sweeps=10, reps=2, passes=1, cache_path=None)),
            ("cd_2pass", lambda: at.tune_batch(b, n_sweeps=10, reps=2, passes=2, cache_path=None)),
            ("class_exhaustive", lambda: at.class_exhaustive_tune_batch(b, n_sweeps=10, reps=2)),
            ("ga_seed0", lambda: at.ga_tune_batch(b, M=10, T=10, n_sweeps=10, reps=2, seed=0)),
            ("ga_seed1", lambda: at.ga_tune_batch(b, M=10, T=10, n_sweeps=10, reps=2, seed=1)))
    for name, search in runs:
        count["n"] = 0
        t0 = time.perf_counter()
        plan = search()
        out[name] = {"value": rate(), "plans_measured": count["n"], "search_s": time.perf_counter() - t0,
                     "plan": {k: plan[k] for k in ("warps", "tile_i", "kdepth")}}
    b.close()
    torch.cuda.empty_cache()

    # a sub-batch small enough to search exhaustively: the grids of the
    # batch with I in {33, 129} and K in {65, 129}, every plan of the space
    sub_ids = [g for g, d in enumerate(dims) if d[0] in (33, 129) and d[2] in (65, 129)]
    sub = [dims[g] for g in sub_ids]
    nsub = sum((I - 2) * (J - 2) * (K - 2) for I, J, K in sub)
    sb = JacobiBatch(sub, "f32", 0.8, stream)
    for q, g in enumerate(sub_ids):
        I, J, K = dims[g]
        sb.upload_tensors(q, ji.himeno_fields_torch(I, J, K, seed=42 + g))
    res = {"grids": len(sub)}

    def sub_rate():
        sb.sweep(sweeps, residuals=False)
        return nsub * sweeps / at.time_call(lambda: sb.sweep(sweeps, residuals=False), 3, stream) / 1e9

    sb.set_plan(0, None, None)
    res["default"] = {"value": sub_rate()}
    subruns = (("joint_exhaustive", lambda: at.joint_exhaustive_tune_batch(sb, n_sweeps=10, reps=2, warps=(8,))),
               ("cd_1pass", lambda: at.tune_batch(sb, n_sweeps=10, reps=2, passes=1, warps=(8,), cache_path=None)),
               ("class_exhaustive", lambda: at.class_exhaustive_tune_batch(sb, n_sweeps=10, reps=2, warps=(8,))),
               ("ga_seed0", lambda: at.ga_tune_batch(sb, M=10, T=10, n_sweeps=10, reps=2, seed=0, warps=(8,))),
               ("ga_seed1", lambda: at.ga_tune_batch(sb, M=10, T=10, n_sweeps=10, reps=2, seed=1, warps=(8,))))
    for name, search in subruns:
        t0 = time.perf_counter()
        plan = search()
        res[name] = {"value": sub_rate(), "search_s": time.perf_counter() - t0,
                     "plan": {k: plan[k] for k in ("warps", "tile_i", "kdepth")}}
        if name == "joint_exhaustive":
            ts = plan["times"]
            res[name].update({"plans_measured": plan["measured"], "best_ms_per_sweep": ts[0] * 1e3,
                              "median_ms_per_sweep": ts[len(ts) // 2] * 1e3, "worst_ms_per_sweep": ts[-1] * 1e3})
    sb.close()
    out["sub_batch_exhaustive"] = res
    torch.cuda.empty_cache()
    return out


def bench_adjoint(args, w, stream, steps=3):
    """n sweeps, then the reverse pass (checkpoint every C) over the last
    `taped` of them, for L = 1/2 |p_T - target|^2."""
    import torch

    import jacobi_inputs as ji
    from paper_2002_12115_gb300 import Jacobi
    I, J, K, prec = w["I"], w["J"], w["K"], w["prec"]
    dev = device_fields(I, J, K)
    target = torch.from_numpy(ji.target_field(I, J, K)).cuda()
    jac = Jacobi(I, J, K, prec, 0.8, stream)
    jac.upload_tensors(dev)
    del dev
    jac.sweep(w["sweeps"] - w["taped"])
    jac.tape_begin(w["C"], w["taped"])
    jac.sweep(w["taped"])
    lam = jac.download_tensor() - target
    del target
    jac.sweep_adjoint(lam)                       # warm-up
    torch.cuda.synchronize()
    a, e = events()
    a.record(stream)
    for _ in range(steps):
        g = jac.sweep_adjoint(lam)
    e.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / steps
    T, C = w["taped"], w["C"]
    recompute = T - (T + C - 1) // C
    nint = n_interior(w)
    bytes_pass = nint * (T * ADJ_BYTES_PER_POINT[prec] + recompute * BYTES_PER_POINT[prec])
    out = {"value": nint * T / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_pass": ms,
           "grid": [I, J, K], "taped_sweeps": T, "checkpoint_every": C, "recomputed_sweeps": recompute,
           "gbs": bytes_pass / (ms * 1e-3) / 1e9, "bytes_per_point_adjoint": ADJ_BYTES_PER_POINT[prec],
           "grad_norms": {k: float(v.norm()) for k, v in g.items()}}
    jac.close()
    del lam, g
    torch.cuda.empty_cache()
    return out


FFT_BYTES_PER_POINT = {"c32": 3 * 2 * 8, "c64": 3 * 2 * 16}   # three passes, each reads and writes every point
# FP64 operations (DADD + DMUL + DFMA, ncu-counted) per point of one spectral
# step of the FP64 FFT (three passes), by grid; the FP64 path is bound by
# GB300's FP64 pipe, not by HBM (profiles/k_fft_pass_512cube.md)
FFT_C64_OPS_PER_POINT = {(512, 512, 512): 96.9}


def bench_fft(args, w, stream, steps=None, warmup=None, e2e=True, parity=True):
    """The spectral step of the 3-D FFT block: every step computes
    inverse(U * exp(-4 pi^2 alpha t |kbar|^2)) and its energy for the next
    time t (three passes, one launch each), U the forward transform of the
    initial field computed once outside the loop.  Gpoint/s = grid points per
    step / time.  e2e: the same step from pinned host memory (copy-in of the
    initial field, forward transform, one spectral step, copy-out of u and of
    the energy) through the C ABI."""
    import numpy as np
    import torch

    import jacobi_inputs as ji
    from paper_2002_12115_gb300 import FFT3
    n1, n2, n3 = w["n"]
    prec, alpha = w["prec"], w["alpha"]
    steps = steps or args.steps
    warmup = warmup or args.warmup
    N = n1 * n2 * n3
    cdt = torch.complex64 if prec == "c32" else torch.complex128
    u0 = ji.fft_field_torch(n1, n2, n3).to(cdt)
    out = {}
    with FFT3(n1, n2, n3, prec, stream) as f:
        U = f.forward(u0)
        u = torch.empty_like(U)
        energy = torch.zeros(1, dtype=torch.float64, device="cuda")
        for k in range(warmup):
            f.evolve(U, alpha, 0.1 * (k + 1), out=u, energy=energy)
        torch.cuda.synchronize()
        a, b = events()
        a.record(stream)
        for k in range(steps):
            f.evolve(U, alpha, 0.1 * (k + 1), out=u, energy=energy)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        gpts = N / (ms * 1e-3) / 1e9
        peak, kind = measured_peak()
        achieved = FFT_BYTES_PER_POINT[prec] * N / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": kind, "bytes_per_point": FFT_BYTES_PER_POINT[prec],
                "kernel": "k_fft_pass (3 passes per step, plus the factor and energy kernels)"}
        ops = FFT_C64_OPS_PER_POINT.get((n1, n2, n3)) if prec == "c64" else None
        if ops:
            ach = ops * N / (ms * 1e-3) / 1e9
            alu = f64_alu_peak_gops()
            roof = {"bound": "alu", "achieved": ach, "peak": alu, "unit": "G FP64 op/s", "frac": ach / alu,
                    "peak_kind": "derived: 2 FP64 ops per SM per clock x 152 SMs x max SM clock",
                    "ops_per_point": ops, "hbm_frac": achieved / peak,
                    "kernel": "k_fft_pass (3 passes per step, plus the factor and energy kernels)"}
        out.update({"value": gpts, "unit": "Gpoint/s (3-D FFT spectral steps)", "ms_per_step": ms,
                    "grid": [n1, n2, n3], "prec": prec, "energy": float(energy.item()),
                    "gflops_5nlogn": 5 * N * np.log2(N) / (ms * 1e-3) / 1e9, "roofline": roof})
        if e2e:
            # two plans on two streams take the steps in turn, so that one
            # step's host copies overlap the other's transforms and copies
            host_u0 = torch.empty(u0.shape, dtype=cdt, pin_memory=True)
            host_u0.copy_(u0)
            s2 = torch.cuda.Stream()
            lanes = []
            for st, plan in ((stream, f), (s2, FFT3(n1, n2, n3, prec, s2))):
                lanes.append({"st": st, "f": plan, "u0": torch.empty_like(u0), "U": torch.empty_like(u0),
                              "u": torch.empty_like(u0), "e": torch.zeros(1, dtype=torch.float64, device="cuda"),
                              "hu": torch.empty(u0.shape, dtype=cdt, pin_memory=True),
                              "he": torch.empty(1, dtype=torch.float64, pin_memory=True)})
            torch.cuda.synchronize()

            def e2e_steps(n):
                for k in range(n):
                    L = lanes[k % 2]
                    with torch.cuda.stream(L["st"]):
                        L["u0"].copy_(host_u0, non_blocking=True)
                        L["f"].forward(L["u0"], out=L["U"])
                        L["f"].evolve(L["U"], alpha, 0.1 * (k + 1), out=L["u"], energy=L["e"])
                        L["hu"].copy_(L["u"], non_blocking=True)
                        L["he"].copy_(L["e"], non_blocking=True)
                    if k >= 1:
                        lanes[(k - 1) % 2]["st"].synchronize()
                lanes[(n - 1) % 2]["st"].synchronize()

            e2e_steps(2)
            t0 = time.perf_counter()
            e2e_steps(steps)
            e2e_ms = (time.perf_counter() - t0) * 1e3 / steps
            lanes[1]["f"].close()
            del lanes
            out["e2e"] = {"value": N / (e2e_ms * 1e-3) / 1e9, "unit": "Gpoint/s (3-D FFT spectral steps)",
                          "h2d_bytes_per_step": N * u0.element_size(), "d2h_bytes_per_step": N * u0.element_size() + 8,
                          "how": "copy-in of the initial field, forward transform, one spectral step, copy-out of "
                                 "the field and the energy, every step; two plans on two streams take the steps "
                                 "in turn"}
        if parity:
            import oracle.fft as fo
            fo.build()
            u0h = u0.cpu().numpy().astype(np.complex128)
            Uh = U.cpu().numpy().astype(np.complex128)
            t_last = 0.1 * steps
            f.evolve(U, alpha, t_last, out=u, energy=energy)
            uh = u.cpu().numpy().astype(np.complex128)
            pts = ji.interior_points(n1 + 2, n2 + 2, n3 + 2, 4, ji.SAMPLE_SEED) - 1     # 4 seeded indices
            errs_U, errs_u = [], []
            kz, ky, kx = (np.fft.fftfreq(n, 1.0 / n) for n in (n3, n2, n1))
            c = -4.0 * np.pi ** 2 * alpha * t_last
            fac = np.exp(c * (kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2))
            W = Uh * fac
            del fac
            for (i, j, k) in pts:
                errs_U.append(abs(fo.point(u0h, (i, j, k)) - Uh[k, j, i]))
                errs_u.append(abs(fo.point(W, (i, j, k), sign=1) / N - uh[k, j, i]))
            e_want = float(np.sum(np.abs(W) ** 2) / N)          # Parseval
            out["parity"] = {"forward_err": max(errs_U) / float(np.abs(Uh).max()),
                             "step_err": max(errs_u) / float(np.abs(uh).max()),
                             "energy_err": abs(float(energy.item()) - e_want) / e_want,
                             "tol": 1e-5 if prec == "c32" else 1e-12,
                             "sample": "4 seeded output points of the forward transform and of the last step, each "
                                       "the FP64 oracle's single-sum DFT over all points; the energy against "
                                       "Parseval's sum |W|^2 / N of the step's spectrum"}
            del u0h, Uh, uh, W
    del u0
    torch.cuda.empty_cache()
    return out


def bench_sweep_latency(w, stream):
    """Per-sweep cost of one launch on a small grid: launches of n = 1 .. 200
    sweeps timed with CUDA events (median of 5), fitted as time = a + b n
    (a: launch and ring start-up, b: one sweep including its grid barrier),
    for the default plan and for plans that give the launch fewer or more
    CTAs (k-depth), and the FP64 arithmetic floor of one sweep."""
    import numpy as np
    import torch

    from paper_2002_12115_gb300 import Jacobi, resolve_plan
    from paper_2002_12115_gb300 import autotune as at
    I, J, K, prec = w["I"], w["J"], w["K"], w["prec"]
    dev = device_fields(I, J, K)
    out = {"grid": [I, J, K], "prec": prec}
    ns = [1, 2, 5, 10, 50, 100, 200]
    plans = {"default": (0, 0, 0)}
    for kd in (1, 2, 4, 8, 16, 32, 63):
        plans[f"kdepth {kd}"] = (0, kd, 0)
    with Jacobi(I, J, K, prec, 0.8, stream) as jac:
        jac.upload_tensors(dev)
        for name, plan in plans.items():
            jac.set_plan(*plan)
            jac.sweep(3)
            jac.residual()
            ts = [at.time_call(lambda: jac.sweep(n), 5, stream) * 1e6 for n in ns]
            b, a = np.polyfit(ns, ts, 1)
            rp = resolve_plan(I, J, K, prec, tile_j=plan[0], kdepth=plan[1], tile_i=plan[2])
            ti, tj, kd = rp["tile_i"], rp["tile_j"], rp["kdepth"]
            items = ((I - 2) // ti + 1) * (-(-(J - 2) // tj)) * (-(-(K - 2) // kd) if kd > 0 else 1)
            out[name] = {"us_per_sweep": b, "launch_us": a, "plan": rp, "work_items": items,
                         "us_at": dict(zip(ns, ts))}
    nint = (I - 2) * (J - 2) * (K - 2)
    out["fp64_alu_floor_us_per_sweep"] = nint * F64_OPS_PER_POINT / (f64_alu_peak_gops() * 1e9) * 1e6
    return out


def run_native(args, w, wname):
    import torch

    from paper_2002_12115_gb300 import lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    args.local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(args.local)
    args.dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", args.local))
        args.dist = dist
    lib()  # fail loudly if the CUDA library is missing
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peak()

    def emit(line):
        if rank == 0:
            print(json.dumps(line, default=str), flush=True)
        if args.dist is not None:
            args.dist.barrier()
            args.dist.destroy_process_group()

    if wname in ("batch", "batch-f64", "batch64"):
        r = bench_batch(args, stream, sweeps=w["sweeps"], steps=args.steps, autotune=not args.no_autotune,
                        tuner=args.tuner, prec=w["prec"], n_grids=w["n_grids"], loops=wname != "batch64")
        value, ms = replica_value(r["points"] * r["sweeps"] / 1e9, r["ms_per_step"], world, args.dist)
        return emit({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                     "warmup": 2, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                     "vs_baseline": None, "dtype": DTYPE[w["prec"]], "data": "synthetic",
                     "config": {"workload": f"{w['n_grids']} grids, dims drawn from {{17,33,49,65,97,129}}, {w['prec']}, 100 "
                                            "sweeps per step in one graph-replayed persistent launch",
                                "l2": f"inputs larger than L2 ({BYTES_PER_POINT[w['prec']] * r['points'] / 1e9:.1f} GB "
                                      "of interior-point bytes swept per sweep)"},
                     "roofline": dict(variant_roofline(w["prec"], r["value"]), traffic=None,
                                      kernel="k_sweep (batched)"),
                     "batch": r, "gpu_launches": args.steps})
    if wname == "tuners":
        r = bench_tuners(stream, sweeps=w["sweeps"])
        return emit({"metric": METRIC + " (512-grid batch under each launch-plan search)",
                     "value": max(v["value"] for k, v in r.items() if "value" in v), "unit": UNIT, "n_gpus": world,
                     "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                     "config": {"workload": "512 grids, dims drawn from {17,33,49,65,97,129}, f32, 100 sweeps; "
                                            "plans searched from scratch"},
                     "searches": r})
    if wname == "sweep-latency":
        r = bench_sweep_latency(w, stream)
        return emit({"metric": "19-pt Jacobi per-sweep latency (us) on a small grid", "value": r["default"]["us_per_sweep"],
                     "unit": "us per sweep", "higher_is_better": False, "n_gpus": world, "dtype": w["prec"],
                     "data": "synthetic", "config": {"workload": f"{w['I']}x{w['J']}x{w['K']} {w['prec']}, launches "
                                                                "of 1..200 sweeps"}, "latency": r})
    if wname.startswith("fft"):
        r = bench_fft(args, w, stream, parity=not args.no_parity, e2e=not args.no_e2e)
        ms = max_over_ranks(r["ms_per_step"], args.dist)
        n1, n2, n3 = w["n"]
        return emit({"metric": "3-D FFT spectral step Gpoint/s & % HBM roofline", "value": r["value"] * world,
                     "unit": r["unit"], "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                     "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                     "dtype": w["prec"], "data": "synthetic",
                     "config": {"workload": f"{n1}x{n2}x{n3} {w['prec']} 3-D FFT spectral steps (heat equation, "
                                            f"alpha {w['alpha']})",
                                "l2": f"inputs larger than L2 ({n1 * n2 * n3 * (8 if w['prec'] == 'c32' else 16) / 1e6:.0f}"
                                      " MB per array); no flush"},
                     "roofline": dict(r["roofline"], traffic=None), "e2e": r.get("e2e"), "parity": r.get("parity"),
                     "gpu_launches": 5 * args.steps, "fft": r})
    if wname.startswith("adjoint"):
        r = bench_adjoint(args, w, stream, steps=args.steps)
        ms = max_over_ranks(r["ms_per_pass"], args.dist)
        return emit({"metric": METRIC + " (adjoint)", "value": r["value"] * world, "unit": UNIT,
                     "n_gpus": world, "steps": args.steps, "warmup": 1, "ms_per_step": ms,
                     "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[w["prec"]],
                     "data": "synthetic",
                     "config": {"workload": f"{w['I']}x{w['J']}x{w['K']} {w['prec']}: {w['sweeps']} sweeps, "
                                            f"reverse pass over the last {w['taped']} with a checkpoint every "
                                            f"{w['C']}"},
                     "roofline": {"bound": "hbm", "achieved": r["gbs"], "peak": peak, "unit": "GB/s",
                                  "frac": r["gbs"] / peak, "peak_kind": peak_kind, "traffic": None,
                                  "kernel": "k_adjoint + recompute k_sweep"},
                     "adjoint": r})

    I, J, K, n, prec = w["I"], w["J"], w["K"], w["sweeps"], w["prec"]
    want_oracle = rank == 0 and not (args.no_parity and args.no_cpu_baseline)
    args.need_host = want_oracle            # FP64 host copies: the oracle's inputs (rank 0)
    s = bench_single(args, w, stream)
    units = n_interior(w) * n * args.steps / 1e9
    value, ms = replica_value(units, s["ms"], world, args.dist)
    e2e = None
    f32_host = prec != "f64"
    if not args.no_e2e:
        e2e_ms = bench_e2e(args, w, s["jac"], stream, s["residual"], s["dev"], f32_host=f32_host)
        e2e, e2e_ms = replica_value(units, e2e_ms, world, args.dist)
    p_gpu = s["p"].cpu().numpy()          # state after the last timed step
    gosa = s["residual"]

    compare = {}
    if not args.no_variants and rank == 0:
        for vp in ("bf16", "f64", "f32"):
            if vp != prec:
                compare[vp] = bench_variant(w, vp, s["dev"], stream, min(n, 30 if vp == "f64" else 200))
        if sweep_split(w, prec, n, args.fuse)[0]:
            # the same grid in single sweeps: the DRAM-bound kernel the passes replace
            compare[prec + "_single_sweeps"] = bench_variant(w, prec, s["dev"], stream, n, fuse=1)
        if prec != "f64":
            try:   # a reported comparison, not a timed figure: an error here is recorded, not raised
                compare["residual_vs_f64_gpu"] = residual_vs_f64(w, s["dev"], stream, n)
            except Exception as e:  # noqa: BLE001
                compare["residual_vs_f64_gpu"] = {"error": str(e)}
    s["jac"].close()
    del s["dev"], s["jac"]
    torch.cuda.empty_cache()
    if not args.no_variants and not args.quick and rank == 0:
        if (I, J, K) == (513, 513, 1025):
            compare["adjoint"] = bench_adjoint(args, WORKLOADS["adjoint"], stream, steps=2)
        c2 = WORKLOADS["config2"]
        if (I, J, K) != (c2["I"], c2["J"], c2["K"]):
            dev2 = device_fields(c2["I"], c2["J"], c2["K"])
            for vp in ("f32", "bf16", "f64"):
                compare["config2_" + vp] = bench_variant(c2, vp, dev2, stream, 200 if vp == "f64" else 1000)
            del dev2
        compare["per_sweep_transfers"] = bench_unhoisted_grid(c2)
        for key in ("fft", "fft-c64"):
            compare[key.replace("-", "_")] = bench_fft(args, WORKLOADS[key], stream, steps=5, warmup=3, e2e=False,
                                                        parity=False)
        compare["batched"] = bench_batch(args, stream, steps=2, autotune=not args.no_autotune)
        torch.cuda.empty_cache()

    # dram_achieved: the ncu bytes of the launch over its live time (below
    # the algorithmic figure when arrays stay in L2)
    roofline = sweep_roofline(w, prec, n, s["launch_ms"], args.fuse)
    roofline.update({"launch_ms": s["launch_ms"], "sweeps_per_launch": n})
    cpu = parity = None
    if want_oracle:
        fields = {k: v.numpy() for k, v in s["host"].items()}
        if not args.no_cpu_baseline:
            gpts, cores, sample = oracle_sample(w, min_seconds=args.cpu_seconds, fields=fields)
            cpu = {"value": gpts, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                   "value_one_core": oracle_one_core(w, fields=fields)}
        if not args.no_parity:
            try:   # reported, not timed: an error here is recorded, not raised
                parity = oracle_parity(w, fields, p_gpu, gosa)
            except Exception as e:  # noqa: BLE001
                parity = {"error": str(e)}
        del fields
    emit({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
        "config": {"workload": workload_name(w), "grid": [I, J, K], "sweeps": n, "prec": prec,
                   "omega": 0.8, "l2": l2_note(w),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "step": "device-side copy-in of resident FP64 inputs, sweeps (one persistent launch), "
                           "residual, copy-out"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "parity": parity,
        "e2e": None if e2e is None else {
            "value": e2e, "unit": UNIT, "h2d_bytes_per_step": 13 * I * J * K * (4 if f32_host else 8),
            "d2h_bytes_per_step": I * J * K * (4 if f32_host else 8) + 8,
            "how": (f"jac_upload_{'f32_' if f32_host else ''}async from pinned host "
                    f"{'FP32' if f32_host else 'FP64'} arrays (the inputs of the {prec} problem), jac_sweep, "
                    f"jac_download_{'f32_' if f32_host else ''}async of the state and the residual, jac_sync; "
                    "two contexts on two streams take the steps in turn")},
        "gpu_launches": args.steps * 15,
        "clocks": s["clocks"],
        "residual": gosa,
        "compare": compare,
    })


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="large")
    ap.add_argument("--tile-j", type=int, default=0)
    ap.add_argument("--kdepth", type=int, default=0)
    ap.add_argument("--tile-i", type=int, default=0)
    ap.add_argument("--fuse", type=int, default=0, choices=(0, 1, 2),
                    help="two-sweep passes for FP32: 0 library's choice, 1 never, 2 always")
    ap.add_argument("--sweeps", type=int, default=0, help="override the workload's sweep count (profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuner", choices=("cd", "ga"), default="cd",
                    help="batch plan search: cached coordinate descent or the genetic algorithm")
    ap.add_argument("--quick", action="store_true", help="skip the adjoint / 129^3-class / batched comparisons")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end steps from host buffers")
    ap.add_argument("--no-parity", action="store_true", help="skip the oracle run on the workload")
    return ap.parse_args(argv)


def main():
    args = parse_args()
    if args.workload == "oracle-configs":       # host cores only, no GPU
        if int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps(oracle_configs()), flush=True)
        return
    w = dict(WORKLOADS[args.workload])
    if args.sweeps:
        w["sweeps"] = args.sweeps
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_native(args, w, args.workload)


if __name__ == "__main__":
    main()
