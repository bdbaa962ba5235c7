"""Asynchronous copy-in and copy-out (jac_upload_async, jac_download_async,
jac_sync) give bitwise the state and residual of the synchronous calls,
including two contexts on two streams that take steps in turn on changing
inputs (the end-to-end pipeline of the benchmark); one pipelined result is
also checked against the FP64 CPU oracle."""
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


def pinned(shape):
    import torch
    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


def pinned_fields(f):
    out = {}
    for k, v in f.items():
        out[k] = pinned(v.shape)
        out[k][...] = v
    return out


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("dims,n", [((33, 33, 65), 7), ((131, 10, 6), 3)])
def test_async_equals_sync(prec, dims, n):
    from paper_2002_12115_gb300 import Jacobi
    I, J, K = dims
    f = ji.himeno_fields(I, J, K, seed=300 + I)
    want_p, want_g = gpu_run(f, n, prec)
    out, res = pinned((K, J, I)), pinned((1,))
    with Jacobi(I, J, K, prec, OMEGA) as jac:
        jac.upload_async(pinned_fields(f))
        jac.sweep(n)
        jac.download_async(out, res)
        jac.sync()
    assert np.array_equal(out, want_p)
    assert res[0] == want_g


def test_pageable_host_arrays():
    """Pageable sources and destinations take the same path (the driver
    copies them before the call returns or at the stream's pace)."""
    from paper_2002_12115_gb300 import Jacobi
    I, J, K, n = 37, 11, 9, 4
    f = ji.himeno_fields(I, J, K, seed=310)
    want_p, want_g = gpu_run(f, n, "f32")
    out, res = np.empty((K, J, I)), np.empty(1)
    with Jacobi(I, J, K, "f32", OMEGA) as jac:
        jac.upload_async(f)
        jac.sweep(n)
        jac.download_async(out, res)
        jac.sync()
    assert np.array_equal(out, want_p) and res[0] == want_g


def test_residual_needs_a_sweep():
    """Asking for the residual before any sweep is JAC_ESTATE; the state alone
    is the rounded p0."""
    from paper_2002_12115_gb300 import JacError, Jacobi
    from paper_2002_12115_gb300.binding import JAC_ESTATE
    I, J, K = 9, 8, 7
    f = ji.himeno_fields(I, J, K, seed=311)
    want_p, _ = gpu_run(f, 0, "f32")
    out, res = pinned((K, J, I)), pinned((1,))
    with Jacobi(I, J, K, "f32", OMEGA) as jac:
        jac.upload_async(pinned_fields(f))
        with pytest.raises(JacError) as e:
            jac.download_async(out, res)
        assert e.value.status == JAC_ESTATE
        jac.download_async(out)
        jac.sync()
    assert np.array_equal(out, want_p)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_two_contexts_in_turn(prec):
    """Seven steps in the benchmark's order (upload of step k, copy-out of step
    k-1, sweeps of step k, wait for step k-1) on two contexts and two streams,
    with the inputs cycling through three seeds, so that each context sees
    different inputs from one step to the next.  Every step's state and
    residual equal, bitwise, the synchronous run of its inputs; the first
    step's also match the oracle."""
    import torch

    from paper_2002_12115_gb300 import Jacobi
    I, J, K, n, steps = 67, 19, 23, 6, 7
    fs = [ji.himeno_fields(I, J, K, seed=s) for s in (320, 321, 322)]
    want = [gpu_run(f, n, prec) for f in fs]
    host = [pinned_fields(f) for f in fs]
    outs, res = [pinned((K, J, I)) for _ in range(2)], [pinned((1,)) for _ in range(2)]
    s2 = torch.cuda.Stream()
    ctxs = (Jacobi(I, J, K, prec, OMEGA), Jacobi(I, J, K, prec, OMEGA, s2))
    got = []

    def finish(k):
        ctxs[k % 2].sync()
        got.append((k, outs[k % 2].copy(), float(res[k % 2][0])))

    try:
        for k in range(steps):
            ctxs[k % 2].upload_async(host[k % 3])
            if k >= 1:
                ctxs[(k - 1) % 2].download_async(outs[(k - 1) % 2], res[(k - 1) % 2])
            ctxs[k % 2].sweep(n)
            if k >= 1:
                finish(k - 1)
        ctxs[(steps - 1) % 2].download_async(outs[(steps - 1) % 2], res[(steps - 1) % 2])
        finish(steps - 1)
    finally:
        for c in ctxs:
            c.close()
    assert [k for k, _, _ in got] == list(range(steps))
    for k, p, g in got:
        wp, wg = want[k % 3]
        assert np.array_equal(p, wp), k
        assert g == wg, k
    op, og = oracle_ref(fs[0], n, prec)
    assert rel_p(got[0][1], op) <= TOL[prec] and rel_g(got[0][2], og) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("dims,n", [((33, 33, 65), 7), ((131, 10, 6), 3)])
def test_fp32_host_copies_equal_fp64_copies_of_the_same_numbers(prec, dims, n):
    """jac_upload_f32_async of FP32 host arrays stores exactly what
    jac_upload_async stores for the same numbers held in FP64, so the state
    and residual are bitwise equal; jac_download_f32_async gives the state
    rounded to FP32 (exact for FP32 storage).  The result also matches the
    oracle on that problem."""
    import torch
    from paper_2002_12115_gb300 import Jacobi
    I, J, K = dims
    f64 = ji.himeno_fields(I, J, K, seed=320 + I)
    f = {k: v.astype(np.float32).astype(np.float64) for k, v in f64.items()}     # FP32 numbers
    want_p, want_g = gpu_run(f, n, prec)
    h32 = {k: torch.from_numpy(v.astype(np.float32)).pin_memory().numpy() for k, v in f.items()}
    out32 = torch.empty((K, J, I), dtype=torch.float32, pin_memory=True).numpy()
    res = pinned((1,))
    with Jacobi(I, J, K, prec, OMEGA) as jac:
        jac.upload_f32_async(h32)
        jac.sweep(n)
        jac.download_f32_async(out32, res)
        jac.sync()
    assert res[0] == want_g
    assert np.array_equal(out32, want_p.astype(np.float32))
    op, og = oracle_ref(f, n, prec)
    assert rel_p(out32.astype(np.float64), op) <= max(TOL[prec], 1e-7) and rel_g(res[0], og) <= TOL[prec]
