"""Full-size parity on the 513 x 513 x 1025 grid (about 270 M points), in the
launch configuration the benchmark times (default plan, one persistent
launch for all 100 sweeps)."""
import numpy as np
import pytest

import jacobi_inputs as ji
from _util import OMEGA, TOL, rel_g, rel_p

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
I, J, K, N_SWEEPS = 513, 513, 1025, 100


@pytest.fixture(scope="module")
def fields():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    import oracle
    oracle.build()
    return ji.himeno_fields(I, J, K)


def test_fp32_full_grid_against_oracle_and_fp64_gpu(fields):
    """FP32 state and residual against the oracle on the same rounded problem
    (full grid, FP32-stored state); the FP32 residual against the FP64 GPU
    run of the same grid is printed (the FP32-state floor, see the readings)."""
    import oracle
    from paper_2002_12115_gb300 import Jacobi
    with Jacobi(I, J, K, "f32", OMEGA) as jac:
        jac.upload(fields)
        jac.sweep(N_SWEEPS)
        g32 = jac.residual()
        p32 = jac.download()
    with Jacobi(I, J, K, "f64", OMEGA) as jac:
        jac.upload(fields)
        jac.sweep(N_SWEEPS)
        g64 = jac.residual()
    fr = oracle.round_inputs(fields, "f32")
    want_p, want_g = oracle.run(fr, N_SWEEPS, OMEGA, state="f32")
    del fr
    ep, eg = rel_p(p32, want_p), rel_g(g32, want_g)
    print(f"513x513x1025 f32: vs oracle p {ep:.3e} residual {eg:.3e}; "
          f"vs FP64 GPU residual {rel_g(g32, g64):.3e} (gosa f32 {g32:.6e}, f64 {g64:.6e})")
    assert ep <= TOL["f32"] and eg <= TOL["f32"]


def test_fp64_sampled_points(fields):
    """FP64 state at 6 seeded interior points, each from the oracle run on
    the box of radius 100 around it (the sweep's dependency cone)."""
    import oracle
    from paper_2002_12115_gb300 import Jacobi
    with Jacobi(I, J, K, "f64", OMEGA) as jac:
        jac.upload(fields)
        jac.sweep(N_SWEEPS)
        p = jac.download()
    pts = ji.interior_points(I, J, K, 6, ji.SAMPLE_SEED)
    want = oracle.sample_after(fields, N_SWEEPS, pts, OMEGA)
    got = np.array([p[k, j, i] for i, j, k in pts])
    assert np.abs(got - want).max() <= 1e-12 * np.abs(p).max(), (got, want)


def test_bf16_sampled_points(fields):
    """BF16-coefficient state at 6 seeded interior points against the oracle
    on the same rounded problem (BF16 coefficients, FP32 state), each from the
    box of radius 100 around the point; the bar is the FP32-state one, far
    inside the workload's 3e-3."""
    import oracle
    from paper_2002_12115_gb300 import Jacobi
    with Jacobi(I, J, K, "bf16", OMEGA) as jac:
        jac.upload(fields)
        jac.sweep(N_SWEEPS)
        p = jac.download()
    pts = ji.interior_points(I, J, K, 6, ji.SAMPLE_SEED, start=18)
    fr = oracle.round_inputs(fields, "bf16")
    want = oracle.sample_after(fr, N_SWEEPS, pts, OMEGA, state="f32")
    del fr
    got = np.array([p[k, j, i] for i, j, k in pts])
    err = float(np.abs(got - want).max() / np.abs(p).max())
    print(f"513x513x1025 bf16 sampled state: max rel err {err:.2e}")
    assert err <= TOL["f32"], (got, want)
