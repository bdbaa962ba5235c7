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


# --------------------------------------------------------------------------
# Genetic-algorithm search, after the paper's offload-pattern search
# (Section 4 and Section 5.1.2): a gene is a bit string; each individual is
# compiled/run and timed; fitness = (time)^(-1/2), which keeps one fast
# individual from taking over the population too early; a run that fails
# (there: did not finish within 3 minutes) counts as a fixed long time
# (there: 1000 s); roulette-wheel selection with the best individual carried
# over unchanged (elite preservation); one-point crossover with probability
# Pc = 0.9 and per-bit mutation with probability Pm = 0.05; the same gene
# recurs often, so measured patterns are cached.  Here a gene encodes a launch
# plan instead of which loops to offload.

GA_PC = 0.9
GA_PM = 0.05
GA_FAIL_SECONDS = 1000.0


class PlanGenome:
    """Bit layout of a batch launch plan: one bit for the warp count, two bits
    per I class for the tile width, three bits per K class for the k-depth
    (values beyond the option list wrap around)."""

    def __init__(self, i_classes, k_classes, widths, kdepths, warps=(8, 4)):
        self.i_classes, self.k_classes = list(i_classes), list(k_classes)
        self.widths, self.kdepths, self.warps = list(widths), list(kdepths), list(warps)
        self.n_bits = 1 + 2 * len(self.i_classes) + 3 * len(self.k_classes)

    @staticmethod
    def _field(bits, start, n):
        v = 0
        for b in bits[start:start + n]:
            v = (v << 1) | int(b)
        return v

    def decode(self, bits) -> dict:
        plan = {"warps": self.warps[self._field(bits, 0, 1) % len(self.warps)], "tile_i": {}, "kdepth": {}}
        pos = 1
        for I in self.i_classes:
            plan["tile_i"][str(I)] = self.widths[self._field(bits, pos, 2) % len(self.widths)]
            pos += 2
        for K in self.k_classes:
            plan["kdepth"][str(K)] = self.kdepths[self._field(bits, pos, 3) % len(self.kdepths)]
            pos += 3
        return plan


def ga_search(n_bits: int, measure, M: int = 10, T: int = 10, pc: float = GA_PC, pm: float = GA_PM,
              seed: int = 0, log=None, on_generation=None):
    """Minimise measure(bits) -> seconds (None or inf = failed run) with the
    paper's GA.  Returns (best_bits, best_time, history); history holds the
    best time of every generation and the number of distinct measurements.
    on_generation(gen, population, times), if given, sees every generation."""
    import numpy as np
    rng = np.random.default_rng(seed)
    cache: dict = {}

    def time_of(bits) -> float:
        key = tuple(int(b) for b in bits)
        if key not in cache:
            t = measure(key)
            cache[key] = GA_FAIL_SECONDS if (t is None or not np.isfinite(t)) else float(t)
        return cache[key]

    pop = [tuple(int(b) for b in rng.integers(0, 2, n_bits)) for _ in range(M)]
    history = []
    best = None
    for gen in range(T):
        times = np.array([time_of(ind) for ind in pop])
        if on_generation:
            on_generation(gen, list(pop), times.copy())
        fit = times ** -0.5
        order = np.argsort(times)
        if best is None or times[order[0]] < best[1]:
            best = (pop[order[0]], float(times[order[0]]))
        history.append({"generation": gen, "best_s": best[1], "measured": len(cache)})
        if log:
            log(f"generation {gen}: best {best[1]:.6f} s, {len(cache)} distinct plans measured")
        if gen == T - 1:
            break
        probs = fit / fit.sum()
        nxt = [pop[order[0]]]                                      # elite preservation
        while len(nxt) < M:
            a, b = (pop[i] for i in rng.choice(M, size=2, p=probs))  # roulette selection
            a, b = list(a), list(b)
            if rng.random() < pc and n_bits > 1:                   # one-point crossover
                cut = int(rng.integers(1, n_bits))
                a[cut:], b[cut:] = b[cut:], a[cut:]
            for child in (a, b):
                for q in range(n_bits):                             # mutation
                    if rng.random() < pm:
                        child[q] ^= 1
                nxt.append(tuple(child))
                if len(nxt) == M:
                    break
        pop = nxt
    return best[0], best[1], history


def ga_tune_batch(batch, M: int = 10, T: int = 10, n_sweeps: int = 10, reps: int = 2, seed: int = 0,
                  kdepths=(4, 8, 16, 32, 64, 12, 24, 48), warps=(8, 4), log=None) -> dict:
    """Per-size-class plan of a JacobiBatch by the GA above, each individual
    timed on the GPU.  Returns the best plan with the search history."""
    dims = batch.dims
    genome = PlanGenome(sorted({d[0] for d in dims}), sorted({d[2] for d in dims}),
                        _tile_widths(batch.prec), kdepths, warps)

    def expand(plan):
        ti = [plan["tile_i"][str(I)] for I, _, _ in dims]
        kd = [min(plan["kdepth"][str(K)], max(K - 2, 1)) for _, _, K in dims]
        return ti, kd

    def measure(bits):
        plan = genome.decode(bits)
        ti, kd = expand(plan)
        try:
            batch.set_plan(plan["warps"], ti, kd)
            batch.sweep(n_sweeps, residuals=False)
        except JacError:
            return None
        return time_call(lambda: batch.sweep(n_sweeps, residuals=False), reps)

    bits, t, history = ga_search(genome.n_bits, measure, M=M, T=T, seed=seed, log=log)
    plan = genome.decode(bits)
    ti, kd = expand(plan)
    batch.set_plan(plan["warps"], ti, kd)
    plan["s_per_sweep"] = t / n_sweeps
    plan["history"] = history
    return plan


# --------------------------------------------------------------------------
# Exhaustive baselines for the searches above.

def _default_plan(dims, widths, warps=8, kdepth=16) -> dict:
    """The starting plan of the coordinate descent: the widest tile that
    wastes the fewest lanes per I class, one k-depth for every K class."""
    return {"warps": warps,
            "tile_i": {str(I): min(widths, key=lambda t: (((I - 2) // t + 1) * t, -t))
                       for I in sorted({d[0] for d in dims})},
            "kdepth": {str(K): kdepth for K in sorted({d[2] for d in dims})}}


def _batch_measure(batch, n_sweeps, reps):
    dims = batch.dims

    def expand(plan):
        ti = [plan["tile_i"][str(I)] for I, _, _ in dims]
        kd = [min(plan["kdepth"][str(K)], max(K - 2, 1)) for _, _, K in dims]
        return ti, kd

    def measure(plan) -> float:
        ti, kd = expand(plan)
        try:
            batch.set_plan(plan["warps"], ti, kd)
            batch.sweep(n_sweeps, residuals=False)
        except JacError:
            return float("inf")
        return time_call(lambda: batch.sweep(n_sweeps, residuals=False), reps)
    return measure, expand


def class_exhaustive_tune_batch(batch, n_sweeps: int = 10, reps: int = 2, kdepths=(4, 8, 16, 32, 64, 12, 24, 48),
                                warps=(8, 4), log=None) -> dict:
    """Exhaustive search per size class: for each warp count, every tile
    width of each I class and every k-depth of each K class is measured with
    all other classes at the default plan; the per-class best choices are
    combined into one plan, which is measured too.  Exact when the batch's
    time is a sum of per-class terms; it measures warps x (widths x I classes
    + depths x K classes) + 1 plans."""
    dims = batch.dims
    widths = _tile_widths(batch.prec)
    measure, expand = _batch_measure(batch, n_sweeps, reps)
    best_plan, best_t, count = None, float("inf"), 0
    for w in warps:
        base = _default_plan(dims, widths, w)
        plan = json.loads(json.dumps(base))
        for I in base["tile_i"]:
            trials = []
            for tw in widths:
                cand = json.loads(json.dumps(base))
                cand["tile_i"][I] = tw
                trials.append((measure(cand), tw))
                count += 1
            plan["tile_i"][I] = min(trials)[1]
        for K in base["kdepth"]:
            trials = []
            for kd in kdepths:
                if kd > max(int(K) - 2, 1):
                    continue
                cand = json.loads(json.dumps(base))
                cand["kdepth"][K] = kd
                trials.append((measure(cand), kd))
                count += 1
            plan["kdepth"][K] = min(trials)[1]
        t = measure(plan)
        count += 1
        if log:
            log(f"warps {w}: combined per-class plan {t / n_sweeps * 1e3:.3f} ms/sweep")
        if t < best_t:
            best_plan, best_t = plan, t
    ti, kd = expand(best_plan)
    batch.set_plan(best_plan["warps"], ti, kd)
    best_plan = dict(best_plan, s_per_sweep=best_t / n_sweeps, measured=count)
    return best_plan


def joint_exhaustive_tune_batch(batch, n_sweeps: int = 5, reps: int = 2, kdepths=(4, 8, 16, 32, 64, 12, 24, 48),
                                warps=(8,), max_plans: int = 4096, log=None) -> dict:
    """Every plan of the batch's plan space (all tile widths of every I class
    times all k-depths of every K class, for each warp count): the true
    optimum the heuristic searches are judged against.  Only for small
    batches (at most max_plans plans)."""
    dims = batch.dims
    widths = _tile_widths(batch.prec)
    i_cl = [str(I) for I in sorted({d[0] for d in dims})]
    k_cl = [str(K) for K in sorted({d[2] for d in dims})]
    k_opts = [[kd for kd in kdepths if kd <= max(int(K) - 2, 1)] or [1] for K in k_cl]
    space = list(product(warps, product(widths, repeat=len(i_cl)), product(*k_opts)))
    if len(space) > max_plans:
        raise ValueError(f"{len(space)} plans: too many for an exhaustive search")
    measure, expand = _batch_measure(batch, n_sweeps, reps)
    results = []
    for w, tws, kds in space:
        plan = {"warps": w, "tile_i": dict(zip(i_cl, tws)), "kdepth": dict(zip(k_cl, kds))}
        results.append((measure(plan), plan))
    results.sort(key=lambda r: r[0])
    t, plan = results[0]
    ti, kd = expand(plan)
    batch.set_plan(plan["warps"], ti, kd)
    if log:
        log(f"{len(results)} plans: best {t / n_sweeps * 1e3:.3f} ms/sweep")
    return dict(plan, s_per_sweep=t / n_sweeps, measured=len(results),
                times=sorted(r[0] / n_sweeps for r in results))
