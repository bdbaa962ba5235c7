"""Seeded input generator: SplitMix64 check values and the workload recipes."""
import json
import os

import numpy as np
import pytest

import jacobi_inputs as ji

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.json")


def test_splitmix64_published_vectors():
    with open(GOLDEN) as fh:
        g = json.load(fh)
    for v in g["vectors"]:
        want = [int(h, 16) for h in v["outputs_hex"]] if "outputs_hex" in v else v["outputs"]
        got = [int(x) for x in ji.splitmix64(v["seed"], 0, len(want))]
        assert got == want
        assert [ji.splitmix64_scalar(v["seed"], n + 1) for n in range(len(want))] == want


def test_stream_is_counter_based():
    full = ji.splitmix64(42, 0, 1000)
    assert np.array_equal(full[300:700], ji.splitmix64(42, 300, 400))
    assert int(full[999]) == ji.splitmix64_scalar(42, 1000)


def test_uniform_range_and_chunked_equality():
    n = (1 << 22) + 12345          # spans two chunks
    u = ji.uniform(7, 0, n, -2.0, 3.0)
    assert u.min() >= -2.0 and u.max() < 3.0
    assert abs(u.mean() - 0.5) < 5e-3
    head = ji.uniform(7, 0, 1000, -2.0, 3.0)
    assert np.array_equal(u[:1000], head)
    z = ji.splitmix64(7, 0, 3)
    want = -2.0 + 5.0 * ((z >> np.uint64(11)).astype(np.float64) / 2.0 ** 53)
    assert np.array_equal(u[:3], want)


def test_field_recipe_order_and_identities():
    I, J, K = 5, 6, 7
    N = I * J * K
    f = ji.himeno_fields(I, J, K)
    for q, name in enumerate(ji.DRAW_ORDER[:-1]):
        lo, hi = ji._RANGES[name]
        assert np.array_equal(f[name].ravel(), ji.uniform(42, q * N, N, lo, hi)), name
    noise = ji.uniform(42, 10 * N, N, -1e-3, 1e-3).reshape(K, J, I)
    kk = (np.arange(K) / (K - 1.0)) ** 2
    assert np.array_equal(f["p"], noise + kk[:, None, None])
    s = f["a0"] + f["a1"] + f["a2"] + f["c0"] + f["c1"] + f["c2"]
    assert np.array_equal(f["a3"], 1.0 / s)
    assert f["bnd"][1:-1, 1:-1, 1:-1].min() == 1.0
    assert f["bnd"].sum() == (I - 2) * (J - 2) * (K - 2)
    for name in ("a0", "a1", "a2", "c0", "c1", "c2"):
        assert 0.95 <= f[name].min() and f[name].max() < 1.05
    for name in ("b0", "b1", "b2"):
        assert -0.02 <= f[name].min() and f[name].max() < 0.02
    assert f["p"].flags["C_CONTIGUOUS"] and f["p"].shape == (K, J, I)


def test_grids_with_distinct_seeds_differ():
    a = ji.himeno_fields(4, 4, 4, seed=42)
    b = ji.himeno_fields(4, 4, 4, seed=43)
    assert not np.array_equal(a["a0"], b["a0"])


def test_too_small_grid_rejected():
    with pytest.raises(ValueError):
        ji.himeno_fields(2, 5, 5)


def test_batch_dims_and_target_modes():
    dims = ji.batch_dims(512)
    assert len(dims) == 512
    flat = [d for t in dims for d in t]
    assert set(flat) == set(ji.BATCH_DIM_CHOICES)
    counts = np.bincount([ji.BATCH_DIM_CHOICES.index(d) for d in flat])
    assert counts.min() > 200          # 1536 draws over 6 values
    modes = ji.target_modes()
    assert len(modes) == 3 and all(1 <= v <= 3 for m in modes for v in m)
    t = ji.target_field(9, 10, 11)
    assert t.shape == (11, 10, 9) and np.abs(t).max() <= 0.3 + 1e-12


def test_fd_points_interior():
    w, a = ji.fd_points(7, 8, 9, 64)
    for pts in (w, a):
        assert pts.shape == (64, 3)
        assert pts[:, 0].min() >= 1 and pts[:, 0].max() <= 5
        assert pts[:, 1].min() >= 1 and pts[:, 1].max() <= 6
        assert pts[:, 2].min() >= 1 and pts[:, 2].max() <= 7


def test_torch_generator_is_bit_identical():
    torch = pytest.importorskip("torch")
    I, J, K = 7, 6, 9
    a = ji.himeno_fields(I, J, K, seed=42)
    b = ji.himeno_fields_torch(I, J, K, seed=42, device="cpu")
    for name in ji.FIELD_NAMES:
        assert np.array_equal(a[name], b[name].numpy()), name
    u = ji.uniform(123, 1000, 5000, -1.0, 1.0)
    v = ji.uniform_torch(123, 1000, 5000, -1.0, 1.0, device="cpu", chunk=777).numpy()
    assert np.array_equal(u, v)


def test_box_generation_equals_slices_of_the_full_grid():
    """himeno_fields_box and target_field_box draw a sub-box of a grid
    directly; they equal, bitwise, the same box cut from the full arrays
    (faces and interior both)."""
    I, J, K = 23, 17, 19
    full = ji.himeno_fields(I, J, K, seed=77)
    tfull = ji.target_field(I, J, K)
    for lo, hi in (((0, 0, 0), (5, 4, 3)), ((7, 3, 11), (23, 17, 19)), ((1, 1, 1), (22, 16, 18))):
        box = ji.himeno_fields_box(I, J, K, lo, hi, seed=77)
        sl = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        for name in ji.FIELD_NAMES:
            assert np.array_equal(box[name], full[name][sl]), name
        assert np.array_equal(ji.target_field_box(I, J, K, lo, hi), tfull[sl])
        assert np.array_equal(ji._box_mask(I, J, K, lo, hi), full["bnd"][sl])
