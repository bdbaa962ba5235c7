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


def test_fitness_is_inverse_square_root_of_time():
    """Roulette weights follow time^(-1/2): with two patterns of 1 s and 4 s
    the faster one is drawn twice as often, not four times."""
    counts = {0: 0, 1: 0}
    rng = np.random.default_rng(0)
    times = np.array([1.0, 4.0])
    fit = times ** -0.5
    for _ in range(20000):
        counts[int(rng.choice(2, p=fit / fit.sum()))] += 1
    assert abs(counts[0] / counts[1] - 2.0) < 0.1


def test_genome_layout_and_wraparound():
    g = PlanGenome([17, 129], [33, 65, 129], [128, 64, 32, 16], [4, 8, 16, 32, 64], (8, 4))
    assert g.n_bits == 1 + 2 * 2 + 3 * 3
    plan = g.decode([1] + [0, 0] + [1, 1] + [0, 0, 0] + [1, 1, 1] + [1, 0, 1])
    assert plan["warps"] == 4
    assert plan["tile_i"] == {"17": 128, "129": 16}
    # 3-bit fields 0, 7, 5 over 5 options wrap to 0, 2, 0
    assert plan["kdepth"] == {"33": 4, "65": 16, "129": 4}
