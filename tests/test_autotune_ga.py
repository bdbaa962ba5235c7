"""The GA plan search (after the paper's offload-pattern GA) on synthetic
fitness landscapes: no GPU involved."""
import numpy as np

from paper_2002_12115_gb300.autotune import GA_FAIL_SECONDS, PlanGenome, ga_search


def test_finds_the_optimum_of_a_separable_landscape():
    target = np.array([1, 0, 1, 1, 0, 0, 1, 0, 1, 1, 0, 1])
    calls = []

    def measure(bits):
        calls.append(bits)
        return 1.0 + np.sum(np.abs(np.array(bits) - target))   # seconds

    bits, t, hist = ga_search(len(target), measure, M=12, T=40, seed=3)
    assert t == 1.0 and np.array_equal(bits, target)
    # elite preservation: the best time never gets worse
    best = [h["best_s"] for h in hist]
    assert all(b2 <= b1 for b1, b2 in zip(best, best[1:]))
    # every distinct pattern is measured once
    assert len(calls) == len(set(calls)) == hist[-1]["measured"]


def test_failed_runs_count_as_the_fixed_penalty():
    def measure(bits):
        return None if bits[0] == 1 else 5.0 - bits[1]

    bits, t, _ = ga_search(3, measure, M=6, T=10, seed=1)
    assert bits[0] == 0 and t == 4.0
    assert GA_FAIL_SECONDS == 1000.0


def test_selection_follows_inverse_square_root_of_time():
    """Drive ga_search itself with crossover and mutation off: the next
    generation is the elite plus roulette draws, so each pattern's share
    grows in proportion to (count x time^-1/2).  With patterns of 1 s and
    4 s, the faster one is drawn twice as often per copy, not four times
    (fitness time^-1) and not equally (no selection)."""
    pops = []

    def measure(bits):
        return 1.0 if bits[0] == 0 else 4.0

    M = 4001
    ga_search(1, measure, M=M, T=2, pc=0.0, pm=0.0, seed=5,
              on_generation=lambda gen, pop, times: pops.append([b[0] for b in pop]))
    n0 = [p.count(0) for p in pops]
    n1 = [p.count(1) for p in pops]
    # generation 1 = the elite (pattern 0) + M - 1 draws with weights n * t^-1/2
    w0, w1 = n0[0] * 1.0, n1[0] * 0.5
    want0 = 1 + (M - 1) * w0 / (w0 + w1)
    assert abs(n0[1] - want0) < 4 * np.sqrt((M - 1) * 0.25)
    # the alternatives are far off
    w0_inv = n0[0] * 1.0
    w1_inv = n1[0] * 0.25
    assert abs(n0[1] - (1 + (M - 1) * w0_inv / (w0_inv + w1_inv))) > 4 * np.sqrt((M - 1) * 0.25)


def test_ga_finds_the_exhaustive_optimum_of_a_plan_landscape():
    """A plan landscape shaped like the batch's (separable per-class costs,
    a warp-count term): the GA with the paper's settings (M = T = 10) and a
    larger budget, against the exhaustive minimum over all decoded plans."""
    from itertools import product
    g = PlanGenome([17, 65, 129], [33, 129], [128, 64, 32, 16], [4, 8, 16, 32, 64, 12, 24, 48], (8, 4))
    pref_w = {"17": 16, "65": 64, "129": 128}
    pref_k = {"33": 8, "129": 16}

    def cost(plan):
        t = 1.0 + (0.1 if plan["warps"] == 4 else 0.0)
        t += sum(0.05 * abs(np.log2(plan["tile_i"][c] / pref_w[c])) for c in pref_w)
        t += sum(0.03 * abs(np.log2(plan["kdepth"][c] / pref_k[c])) for c in pref_k)
        return t

    best = min(cost(g.decode(bits)) for bits in product((0, 1), repeat=g.n_bits))
    _, t_small, _ = ga_search(g.n_bits, lambda b: cost(g.decode(b)), M=10, T=10, seed=0)
    _, t_big, _ = ga_search(g.n_bits, lambda b: cost(g.decode(b)), M=30, T=40, seed=0)
    assert best == 1.0
    assert t_big <= t_small and t_big <= best + 0.06      # within one step of one class's choice
    assert t_small >= best


def test_genome_layout_and_wraparound():
    g = PlanGenome([17, 129], [33, 65, 129], [128, 64, 32, 16], [4, 8, 16, 32, 64], (8, 4))
    assert g.n_bits == 1 + 2 * 2 + 3 * 3
    plan = g.decode([1] + [0, 0] + [1, 1] + [0, 0, 0] + [1, 1, 1] + [1, 0, 1])
    assert plan["warps"] == 4
    assert plan["tile_i"] == {"17": 128, "129": 16}
    # 3-bit fields 0, 7, 5 over 5 options wrap to 0, 2, 0
    assert plan["kdepth"] == {"33": 4, "65": 16, "129": 4}
