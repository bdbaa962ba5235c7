"""GPU forward sweep (through the C ABI) against the FP64 CPU oracle.

Bars: FP64 1e-12, FP32 1e-5, BF16-coefficient storage 3e-3, relative, on the
state (normwise, max|dp| / max|p|) and on the residual of the last sweep.
The FP32 and BF16 paths are compared with the oracle run on the same rounded
inputs with its state rounded to FP32 after every sweep (the problem those
paths store); the error against the plain FP64 problem is printed.
"""
import numpy as np
import pytest

import jacobi_inputs as ji
from _util import OMEGA, TOL, gpu_run, oracle_ref, rel_g, rel_p

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    import oracle
    oracle.build()


SMALL = [((3, 3, 3), 1), ((4, 4, 4), 3), ((5, 6, 7), 7), ((17, 9, 11), 5), ((37, 11, 9), 4),
         ((130, 9, 12), 3), ((131, 10, 6), 2), ((67, 19, 23), 6), ((9, 40, 5), 2)]
# (tile_j, kdepth, tile_i); tile_i 0 = the widest tile for that tile_j
# kdepth -1: balanced ranges of tile-planes (FP64)
PLANS = {"f64": [None, (4, 1, 0), (8, 3, 0), (8, 1000, 0), (32, 2, 16), (8, -1, 0), (16, -1, 32), (4, -1, 0)],
         "f32": [None, (4, 1, 0), (8, 3, 0), (8, 1000, 0), (32, 2, 32), (64, 3, 16)],
         "bf16": [None, (4, 1, 0), (16, 3, 0), (8, 1000, 0), (64, 2, 32)]}


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("dims,n", SMALL)
def test_small_ragged_grids(prec, dims, n):
    I, J, K = dims
    f = ji.himeno_fields(I, J, K, seed=100 + I + J + K)
    want_p, want_g = oracle_ref(f, n, prec)
    for plan in PLANS[prec]:
        p, g = gpu_run(f, n, prec, plan)
        assert rel_p(p, want_p) <= TOL[prec], (plan, rel_p(p, want_p))
        assert rel_g(g, want_g) <= TOL[prec], (plan, rel_g(g, want_g))


def test_config1_fp64_200_sweeps():
    """33 x 33 x 65, FP64, 200 sweeps: 1e-12 in p and in the residual."""
    f = ji.himeno_fields(33, 33, 65)
    want_p, want_g = oracle_ref(f, 200, "f64")
    p, g = gpu_run(f, 200, "f64")
    print(f"config1 f64: p err {rel_p(p, want_p):.3e} residual err {rel_g(g, want_g):.3e} gosa {g:.6e}")
    assert rel_p(p, want_p) <= 1e-12
    assert rel_g(g, want_g) <= 1e-12


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["f32", "bf16", "f64"])
def test_config2_1000_sweeps(prec):
    """129 x 129 x 257, 1000 resident sweeps, each precision."""
    import oracle
    f = ji.himeno_fields(129, 129, 257)
    want_p, want_g = oracle_ref(f, 1000, prec)
    p, g = gpu_run(f, 1000, prec)
    ep, eg = rel_p(p, want_p), rel_g(g, want_g)
    msg = f"config2 {prec}: vs stored-precision oracle p {ep:.3e} residual {eg:.3e}"
    if prec != "f64":
        p64, g64 = oracle.run(f, 1000, OMEGA)
        msg += f"; vs FP64 problem p {rel_p(p, p64):.3e} residual {rel_g(g, g64):.3e}"
    print(msg)
    assert ep <= TOL[prec] and eg <= TOL[prec], msg


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_constant_fixed_point_exact(prec):
    """a = 1.5, 1.5, 1.5 / c = 1.5, 1, 1, a3 = 1/8, wrk1 = 0, p = 0.75: every
    operation is exact in every precision, so p stays bitwise and gosa = 0."""
    I, J, K = 41, 13, 17
    shape = (K, J, I)
    rng = np.random.default_rng(0)
    f = {n: np.full(shape, v) for n, v in (("a0", 1.5), ("a1", 1.5), ("a2", 1.5), ("c0", 1.5),
                                          ("c1", 1.0), ("c2", 1.0), ("a3", 0.125))}
    for n in ("b0", "b1", "b2"):
        f[n] = rng.uniform(-0.02, 0.02, shape)
    f["wrk1"] = np.zeros(shape)
    f["bnd"] = ji.interior_mask(I, J, K)
    f["p"] = np.full(shape, 0.75)
    p, g = gpu_run(f, 9, prec)
    assert np.array_equal(p, f["p"]) and g == 0.0


def test_sine_mode_closed_form_fp64():
    """Discrete sine mode with a_d = c_d, b = 0, wrk1 = 0: p_n = g^n p0 and
    gosa_n = (1 - lambda)^2 g^(2(n-1)) sum p0^2 (see the oracle pins)."""
    I, J, K = 65, 33, 49
    alphas = (1.0, 1.3, 0.7)
    shape = (K, J, I)
    f = {}
    for d, (a, c) in enumerate((("a0", "c0"), ("a1", "c1"), ("a2", "c2"))):
        f[a] = np.full(shape, alphas[d])
        f[c] = np.full(shape, alphas[d])
    for n in ("b0", "b1", "b2", "wrk1"):
        f[n] = np.zeros(shape)
    f["a3"] = np.full(shape, 1.0 / (2 * sum(alphas)))
    f["bnd"] = ji.interior_mask(I, J, K)
    k, j, i = np.meshgrid(np.arange(K), np.arange(J), np.arange(I), indexing="ij")
    th = (np.pi * 2 / (I - 1), np.pi * 1 / (J - 1), np.pi * 3 / (K - 1))
    p0 = np.sin(th[0] * i) * np.sin(th[1] * j) * np.sin(th[2] * k) * f["bnd"]
    f["p"] = p0
    lam = sum(a * np.cos(t) for a, t in zip(alphas, th)) / sum(alphas)
    gf = 1 - OMEGA * (1 - lam)
    n = 25
    p, g = gpu_run(f, n, "f64")
    assert np.abs(p - gf ** n * p0).max() <= 1e-13
    want = (1 - lam) ** 2 * gf ** (2 * (n - 1)) * np.sum(p0[1:-1, 1:-1, 1:-1] ** 2)
    assert abs(g - want) <= 1e-12 * want


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_mask_invariant_and_faces(prec):
    I, J, K = 70, 21, 19
    f = ji.himeno_fields(I, J, K, seed=77)
    holes = np.random.default_rng(2).random(f["bnd"].shape) < 0.15
    f["bnd"] = np.where(holes, 0.0, f["bnd"])
    p, g = gpu_run(f, 11, prec)
    import oracle
    frozen = f["bnd"] == 0.0
    stored = oracle.round_inputs(f, prec)["p"]
    assert np.array_equal(p[frozen], stored[frozen])
    want_p, want_g = oracle_ref(f, 11, prec)
    assert rel_p(p, want_p) <= TOL[prec] and rel_g(g, want_g) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
def test_bitwise_reproducible_and_plan_invariant_state(prec):
    """Two runs give bitwise the same state and residual; other launch plans
    give bitwise the same state (the per-point arithmetic does not depend on
    the tiling) and the same residual to reduction-order rounding."""
    f = ji.himeno_fields(97, 65, 33, seed=5)
    p1, g1 = gpu_run(f, 13, prec)
    p2, g2 = gpu_run(f, 13, prec)
    assert np.array_equal(p1, p2) and g1 == g2
    plans = [(4, 2), (16 if prec == "bf16" else 8, 7), (32, 5, 16)]
    if prec == "f64":
        plans += [(8, -1), (32, -1, 16), (8, 40)]
    for plan in plans:
        p3, g3 = gpu_run(f, 13, prec, plan)
        assert np.array_equal(p1, p3)
        assert abs(g3 - g1) <= 1e-13 * g1


def test_zero_sweeps_and_omega_zero():
    f = ji.himeno_fields(20, 21, 22, seed=3)
    p, _ = gpu_run(f, 0, "f32")
    assert np.array_equal(p, f["p"].astype(np.float32).astype(np.float64))
    p, g = gpu_run(f, 4, "f64", omega=0.0)
    assert np.array_equal(p, f["p"]) and g > 0


def test_api_errors():
    from paper_2002_12115_gb300 import JacError, Jacobi
    with Jacobi(9, 9, 9, "f32") as jac:
        with pytest.raises(JacError, match="JAC_ESTATE"):
            jac.sweep(1)
        f = ji.himeno_fields(9, 9, 9)
        jac.upload(f)
        with pytest.raises(JacError, match="JAC_ESTATE"):
            jac.residual()
        with pytest.raises(JacError, match="JAC_EINVAL"):
            jac.set_plan(5, 0)
        with pytest.raises(JacError, match="JAC_EINVAL"):
            jac.set_plan(16, 0, 128)       # 16 warps: BF16 coefficients only
        with pytest.raises(JacError, match="JAC_EINVAL"):
            jac.set_plan(8, 0, 48)         # not a power of two
        with pytest.raises(JacError, match="JAC_EINVAL"):
            jac.set_plan(8, -2)            # -1 (balanced) is the only negative depth
        with pytest.raises(JacError, match="JAC_EINVAL"):
            jac.set_plan(8, -1)            # balanced ranges: FP64 storage only
        jac.set_plan(0, 0)
        with pytest.raises(JacError, match="JAC_EINVAL"):
            jac.sweep(-1)
        jac.sweep(2)
        assert jac.count() == 2 and jac.residual() > 0


def test_unhoisted_matches_hoisted():
    """Per-sweep copy-in / copy-out gives the same state when the state is
    representable (FP64 storage)."""
    from paper_2002_12115_gb300 import Jacobi
    f = ji.himeno_fields(33, 17, 21, seed=8)
    p_h, g_h = gpu_run(f, 5, "f64")
    with Jacobi(33, 17, 21, "f64") as jac:
        ph = f["p"].copy()
        jac.sweep_unhoisted(5, f, ph)
        g = jac.residual()
    assert np.array_equal(ph, p_h) and g == g_h
