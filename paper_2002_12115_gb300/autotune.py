"""Launch-plan autotuner: choose tile shapes and k-block depths by measuring.

The paper finds which loop statements to offload by trying candidate offload
patterns on the target machine and keeping the fastest (a genetic algorithm
whose fitness is the measured run time, Sections 3.2 and 4); a loop's
suitability cannot be predicted, only measured.  This module applies the
same principle to the sweep's launch plan: candidate plans are run on the
GPU, timed with CUDA events (median of several repetitions), and the fastest
is kept and cached.

  * ``tune_grid``  -- one grid: tile width x rows x k-block depth;
  * ``tune_batch`` -- a batch: warp count for the launch, then coordinate
    descent over a tile width per size class (grid I) and a k-block depth
    per size class (grid K).

Results are cached in a JSON file keyed by GPU name, precision and workload
(by default autotune_cache.json next to this module).
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
from itertools import product

from .binding import JacError

# plans measured on this project's GPUs ship with the package; set
# JAC_AUTOTUNE_CACHE to keep a cache elsewhere
CACHE_PATH = os.environ.get("JAC_AUTOTUNE_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json"))


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def _load_cache(path: str) -> dict:
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store_cache(path: str, cache: dict) -> None:
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def time_call(fn, reps: int = 3, stream=None) -> float:
    """Median wall time of fn() in seconds, bracketed by CUDA events."""
    import torch
    s = stream or torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        times.append(a.elapsed_time(b) * 1e-3)
    return statistics.median(times)


def _tile_widths(prec: str) -> list[int]:
    return [64, 32, 16] if prec == "f64" else [128, 64, 32, 16]


def tune_grid(jac, n_sweeps: int = 20, reps: int = 3, kdepths=(2, 4, 8, 16, 32, 64), warps=(4, 8, 16),
              cache_path: str | None = CACHE_PATH) -> dict:
    """Best (tile_i, tile_j, kdepth) of a Jacobi context by measurement.
    The context must hold uploaded fields; its state advances while tuning."""
    key = f"grid|{_gpu_name()}|{jac.prec}|{jac.I}x{jac.J}x{jac.K}"
    cache = _load_cache(cache_path) if cache_path else {}
    if key in cache:
        best = cache[key]
        jac.set_plan(best["tile_j"], best["kdepth"], best["tile_i"])
        return best
    full = 64 if jac.prec == "f64" else 128
    trials = []
    for ti, w, kd in product(_tile_widths(jac.prec), warps, kdepths):
        if kd > jac.K - 2 and kd != kdepths[0]:
            continue
        plan = (w * (full // ti), kd, ti)
        try:
            jac.set_plan(*plan)
        except JacError:
            continue
        jac.sweep(1)  # warm-up of this shape
        t = time_call(lambda: jac.sweep(n_sweeps), reps)
        trials.append((t, plan))
    trials.sort()
    t, (tj, kd, ti) = trials[0]
    best = {"tile_i": ti, "tile_j": tj, "kdepth": kd, "s_per_sweep": t / n_sweeps, "trials": len(trials)}
    jac.set_plan(tj, kd, ti)
    if cache_path:
        cache[key] = best
        _store_cache(cache_path, cache)
    return best


def tune_batch(batch, n_sweeps: int = 10, reps: int = 3, passes: int = 2, kdepths=(4, 8, 16, 32, 64),
               warps=(8, 4), cache_path: str | None = CACHE_PATH, log=None) -> dict:
    """Per-size-class plan of a JacobiBatch by coordinate descent on measured
    time: tile width per grid I, k-block depth per grid K, warps per launch.
    The batch must hold uploaded fields; its state advances while tuning."""
    dims = batch.dims
    sig = ",".join(f"{I}x{J}x{K}" for I, J, K in dims)
    key = f"batch|{_gpu_name()}|{batch.prec}|{len(dims)}|{hashlib.sha1(sig.encode()).hexdigest()[:12]}"
    cache = _load_cache(cache_path) if cache_path else {}
    i_classes = sorted({d[0] for d in dims})
    k_classes = sorted({d[2] for d in dims})

    def expand(plan):
        ti = [plan["tile_i"][str(I)] for I, _, _ in dims]
        kd = [min(plan["kdepth"][str(K)], max(K - 2, 1)) for _, _, K in dims]
        return ti, kd

    def measure(plan) -> float:
        ti, kd = expand(plan)
        try:
            batch.set_plan(plan["warps"], ti, kd)
            batch.sweep(n_sweeps, residuals=False)   # capture + warm-up
        except JacError:
            return float("inf")
        return time_call(lambda: batch.sweep(n_sweeps, residuals=False), reps)

    if key in cache:
        plan = cache[key]
        ti, kd = expand(plan)
        batch.set_plan(plan["warps"], ti, kd)
        return plan

    widths = _tile_widths(batch.prec)
    best_plan = None
    best_t = float("inf")
    for w in warps:
        # start: widest tile that wastes the fewest lanes, k-depth 16
        plan = {"warps": w,
                "tile_i": {str(I): min(widths, key=lambda t: (((I - 2) // t + 1) * t, -t)) for I in i_classes},
                "kdepth": {str(K): 16 for K in k_classes}}
        t_cur = measure(plan)
        for _ in range(passes):
            for I in i_classes:
                for tw in widths:
                    if tw == plan["tile_i"][str(I)]:
                        continue
                    cand = json.loads(json.dumps(plan))
                    cand["tile_i"][str(I)] = tw
                    t = measure(cand)
                    if t < t_cur:
                        plan, t_cur = cand, t
            for K in k_classes:
                for kd in kdepths:
                    if kd == plan["kdepth"][str(K)] or kd > max(K - 2, 1):
                        continue
                    cand = json.loads(json.dumps(plan))
                    cand["kdepth"][str(K)] = kd
                    t = measure(cand)
                    if t < t_cur:
                        plan, t_cur = cand, t
        if log:
            log(f"warps {w}: {t_cur / n_sweeps * 1e3:.3f} ms/sweep")
        if t_cur < best_t:
            best_plan, best_t = plan, t_cur
    best_plan = dict(best_plan)
    best_plan["s_per_sweep"] = best_t / n_sweeps
    ti, kd = expand(best_plan)
    batch.set_plan(best_plan["warps"], ti, kd)
    if cache_path:
        cache[key] = best_plan
        _store_cache(cache_path, cache)
    return best_plan
