"""Batched persistent sweeps (one launch for many uneven grids, replayed from
a CUDA graph) and row folding, against the single-grid path and the oracle."""
import numpy as np
import pytest

import jacobi_inputs as ji
from _util import OMEGA, TOL, gpu_run, oracle_ref, rel_g, rel_p, residual_ok

pytestmark = pytest.mark.gpu

DIMS = [(17, 17, 17), (33, 17, 49), (17, 65, 33), (49, 33, 17), (97, 17, 33), (129, 33, 17),
        (65, 49, 19), (33, 129, 9), (20, 9, 13), (3, 3, 3), (5, 40, 6)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    import oracle
    oracle.build()


def make_batch(dims, prec, seed0=42):
    from paper_2002_12115_gb300 import JacobiBatch
    b = JacobiBatch(dims, prec, OMEGA)
    fields = []
    for g, (I, J, K) in enumerate(dims):
        f = ji.himeno_fields(I, J, K, seed=seed0 + g)
        b.upload(g, f)
        fields.append(f)
    return b, fields


@pytest.mark.parametrize("prec", ["f32", "f64", "bf16"])
def test_batch_matches_single_grid_and_oracle(prec):
    """One launch for all grids gives each grid bitwise the state of its own
    single-grid run (same per-grid plan) and matches the oracle."""
    n = 7
    b, fields = make_batch(DIMS, prec)
    res = b.sweep(n)
    for g, f in enumerate(fields):
        tile_i, tile_j, kd = b.grid_plan(g)
        p_single, g_single = gpu_run(f, n, prec, (tile_j, kd, tile_i))
        p = b.download(g)
        assert np.array_equal(p, p_single), g
        assert abs(res[g] - g_single) <= 1e-13 * g_single, g
        want_p, want_g = oracle_ref(f, n, prec)
        n_int = np.prod([d - 2 for d in DIMS[g]])
        assert rel_p(p, want_p) <= TOL[prec] and residual_ok(res[g], want_g, prec, n_int), g
    b.close()


def test_graph_replay_and_buffer_parity():
    """Consecutive calls (the second replays the captured graph; odd counts
    flip the state buffer) continue the same iteration."""
    b, fields = make_batch(DIMS[:6], "f32")
    b.sweep(3)
    b.sweep(3)
    r = b.sweep(4)
    for g, f in enumerate(fields):
        tile_i, tile_j, kd = b.grid_plan(g)
        p_single, g_single = gpu_run(f, 10, "f32", (tile_j, kd, tile_i))
        assert np.array_equal(b.download(g), p_single)
        assert abs(r[g] - g_single) <= 1e-13 * g_single
    assert b.info()["sweeps"] == 10
    b.close()


@pytest.mark.parametrize("per_sweep", [False, True])
def test_loop_of_per_grid_launches_matches(per_sweep):
    b1, fields = make_batch(DIMS, "f32")
    b2, _ = make_batch(DIMS, "f32")
    r1 = b1.sweep(5)
    r2 = b2.sweep_loop(5, per_sweep=per_sweep)
    for g in range(len(DIMS)):
        assert np.array_equal(b1.download(g), b2.download(g))
        assert abs(r1[g] - r2[g]) <= 1e-13 * r2[g]
    b1.close()
    b2.close()


def test_per_grid_plans_do_not_change_the_state():
    rng = np.random.default_rng(0)
    b1, _ = make_batch(DIMS, "f32")
    b2, _ = make_batch(DIMS, "f32")
    ti = [int(rng.choice([128, 64, 32, 16])) for _ in DIMS]
    kd = [int(rng.integers(1, 20)) for _ in DIMS]
    b2.set_plan(4, ti, kd)
    b1.sweep(6)
    b2.sweep(6)
    for g in range(len(DIMS)):
        assert np.array_equal(b1.download(g), b2.download(g))
    b1.close()
    b2.close()


@pytest.mark.parametrize("prec,plans", [("f32", [(32, 3, 32), (64, 2, 16), (16, 5, 64), (8, 2, 128)]),
                                        ("f64", [(32, 3, 16), (8, 4, 32), (8, 2, 64)]),
                                        ("bf16", [(64, 3, 32), (32, 2, 64), (16, 4, 128)])])
def test_row_folding_single_grid(prec, plans):
    """Narrow tall tiles (several rows per warp) give the same state."""
    f = ji.himeno_fields(37, 45, 21, seed=4)
    ref, gref = gpu_run(f, 5, prec)
    want_p, want_g = oracle_ref(f, 5, prec)
    for plan in plans:
        p, g = gpu_run(f, 5, prec, plan)
        assert np.array_equal(p, ref), plan
        assert rel_p(p, want_p) <= TOL[prec] and rel_g(g, want_g) <= TOL[prec]


def test_autotuner_small_batch(tmp_path):
    from paper_2002_12115_gb300 import autotune
    b, _ = make_batch(DIMS[:5], "f32")
    ref, _ = make_batch(DIMS[:5], "f32")
    plan = autotune.tune_batch(b, n_sweeps=2, reps=1, passes=1, cache_path=str(tmp_path / "c.json"))
    assert plan["warps"] in (4, 8) and (tmp_path / "c.json").exists()
    n_done = b.info()["sweeps"]
    ref.sweep(n_done)
    for g in range(5):
        assert np.array_equal(b.download(g), ref.download(g))
    b.close()
    ref.close()


def test_ga_and_exhaustive_plan_searches_on_a_small_batch():
    """The paper's GA (ga_tune_batch), the per-class exhaustive search and
    the joint exhaustive search (every plan of the space) run on the GPU on
    a small batch of two I classes and two K classes.  Every plan they pick
    is valid, the joint optimum is no slower than the others' plans beyond
    timing noise, and the batch's state after all the tuning sweeps equals,
    bitwise, that of a batch swept with the default plan (a launch plan
    never changes results)."""
    from paper_2002_12115_gb300 import autotune
    dims = [(17, 33, 33), (33, 17, 33), (17, 17, 65), (33, 33, 65), (33, 21, 65)]
    b, _ = make_batch(dims, "f32")
    ref, _ = make_batch(dims, "f32")
    kd = (4, 8, 16, 32)
    joint = autotune.joint_exhaustive_tune_batch(b, n_sweeps=2, reps=1, kdepths=kd, warps=(8,))
    assert joint["measured"] == 4 * 4 * 3 * 4          # widths^2 x depths(K=33) x depths(K=65)
    ga = autotune.ga_tune_batch(b, M=6, T=4, n_sweeps=2, reps=1, kdepths=kd, warps=(8,))
    cls = autotune.class_exhaustive_tune_batch(b, n_sweeps=2, reps=1, kdepths=kd, warps=(8,))
    for plan in (joint, ga, cls):
        assert set(plan["tile_i"]) == {"17", "33"} and set(plan["kdepth"]) == {"33", "65"}
        assert all(v in (128, 64, 32, 16) for v in plan["tile_i"].values())
    assert joint["s_per_sweep"] <= 1.5 * min(ga["s_per_sweep"], cls["s_per_sweep"])
    assert len(ga["history"]) == 4
    n_done = b.info()["sweeps"]
    ref.sweep(n_done)
    for g in range(len(dims)):
        assert np.array_equal(b.download(g), ref.download(g)), g
    b.close()
    ref.close()


@pytest.mark.slow
def test_config4_full_batch():
    """512 grids with dims drawn from {17, ..., 129}, 100 FP32 sweeps in one
    launch: bitwise equal to per-grid launches, and every one of the 512
    grids (state and residual) matched with the oracle on its own rounded
    problem."""
    import torch
    from paper_2002_12115_gb300 import JacobiBatch
    dims = ji.batch_dims(512)
    b1 = JacobiBatch(dims, "f32", OMEGA)
    b2 = JacobiBatch(dims, "f32", OMEGA)
    for g, (I, J, K) in enumerate(dims):
        t = ji.himeno_fields_torch(I, J, K, seed=42 + g)
        b1.upload_tensors(g, t)
        b2.upload_tensors(g, t)
    r1 = b1.sweep(100)
    r2 = b2.sweep_loop(100)
    torch.cuda.synchronize()
    for g in range(512):
        assert torch.equal(b1.download_tensor(g), b2.download_tensor(g)), g
    assert np.all(np.abs(r1 - r2) <= 1e-13 * r2)
    worst = (0.0, 0.0)
    for g, (I, J, K) in enumerate(dims):
        f = ji.himeno_fields(I, J, K, seed=42 + g)
        want_p, want_g = oracle_ref(f, 100, "f32")
        ep, eg = rel_p(b1.download(g), want_p), rel_g(r1[g], want_g)
        assert ep <= TOL["f32"] and eg <= TOL["f32"], (g, ep, eg)
        worst = (max(worst[0], ep), max(worst[1], eg))
    print(f"512 grids against the oracle: worst p err {worst[0]:.2e}, residual err {worst[1]:.2e}")
    b1.close()
    b2.close()
