"""Borrowed contexts (jac_create_borrowed): the caller, here torch, owns every
byte of device memory the hoisted path uses -- the fourteen storage arrays
and one workspace holding the sweep scratch, the staging array and the
checkpoint tape.  The library allocates nothing: across upload, sweeps,
tape and the reverse pass the device's free memory moves only by what torch
itself reserves, and torch's allocated bytes are exactly the buffers the
context was given.  Results match the oracle (forward) and the reverse-mode
oracle (gradients)."""
import numpy as np
import pytest

import jacobi_inputs as ji
from _util import TOL, oracle_ref, rel_g, rel_p

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    import oracle
    oracle.build()
    import paper_2002_12115_gb300 as p
    return p


def _run(pkg, f, target, prec, T, C):
    import torch
    K, J, I = f["p"].shape
    jac = pkg.Jacobi(I, J, K, prec, tape=(C, T))
    jac.upload(f)
    jac.tape_begin(C, T)
    jac.sweep(T)
    g_res = jac.residual()
    p = jac.download()
    lam = torch.from_numpy(p - target).cuda()
    grads = jac.sweep_adjoint(lam, coef_grads=True)
    torch.cuda.synchronize()
    return jac, p, g_res, {k: v.cpu().numpy() for k, v in grads.items()}


def _round512(n):
    return (n + 511) // 512 * 512


def test_borrowed_path_allocates_nothing_and_matches_oracles(pkg):
    import torch
    import oracle
    I, J, K, T, C = 37, 29, 23, 6, 2
    f = ji.himeno_fields(I, J, K, seed=500)
    target = ji.target_field(I, J, K)
    # warm-up: loads the kernels (lazy module loading takes device memory once)
    jac, *_ = _run(pkg, f, target, "f64", T, C)
    jac.close()
    del jac
    torch.cuda.synchronize()

    free0 = torch.cuda.mem_get_info()[0]
    res0, alloc0 = torch.cuda.memory_reserved(), torch.cuda.memory_allocated()
    jac = pkg.Jacobi(I, J, K, "f64", tape=(C, T))
    # torch holds exactly the buffers handed to the library
    want = [pkg.field_bytes(I, J, K, "f64", 0)] * 2 + [pkg.field_bytes(I, J, K, "f64", q) for q in range(1, 13)]
    want.append(pkg.ctx_workspace_size(I, J, K, "f64", tape=(C, T)))
    assert jac.device_bytes() == sum(want)
    assert torch.cuda.memory_allocated() - alloc0 == sum(_round512(b) for b in want)
    jac.close()
    jac, p, g_res, grads = _run(pkg, f, target, "f64", T, C)
    free1 = torch.cuda.mem_get_info()[0]
    res1 = torch.cuda.memory_reserved()
    # every change of free device memory is torch's own reservation
    assert abs((free0 - free1) - (res1 - res0)) <= 2 << 20, (free0 - free1, res1 - res0)
    jac.close()

    op, og = oracle_ref(f, T, "f64")
    assert rel_p(p, op) <= TOL["f64"] and rel_g(g_res, og) <= TOL["f64"]
    want_g = oracle.adjoint(f, T, target, 0.8, coef_grads=True)
    for key in ("g_wrk1", "g_a3", "g_p0", "g_a0", "g_b1", "g_c2"):
        err = np.abs(grads[key] - want_g[key]).max() / np.abs(want_g[key]).max()
        assert err <= 1e-10, (key, err)


def test_borrowed_workspace_grows_for_async_upload_and_longer_tape(pkg):
    """A borrowed context sized without asynchronous staging or tape gets a
    larger torch workspace when a call needs one (jac_set_workspace); the
    results equal those of a context that owns its memory, bit for bit."""
    import torch
    I, J, K, T, C = 66, 19, 17, 5, 3
    f = ji.himeno_fields(I, J, K, seed=501)
    pinned = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in f.items()}
    out = {}
    for owned in (True, False):
        with pkg.Jacobi(I, J, K, "f32", owned=owned) as jac:
            jac.upload_async(pinned)
            jac.tape_begin(C, T)
            jac.sweep(T)
            p = np.zeros((K, J, I))
            res = np.zeros(1)
            jac.download_async(p, res)
            jac.sync()
            lam = torch.from_numpy(p - ji.target_field(I, J, K)).cuda()
            g = jac.sweep_adjoint(lam)
            out[owned] = (p, res[0], {k: v.cpu().numpy() for k, v in g.items()})
    assert np.array_equal(out[True][0], out[False][0]) and out[True][1] == out[False][1]
    for k in out[True][2]:
        assert np.array_equal(out[True][2][k], out[False][2][k]), k
    op, og = oracle_ref(f, T, "f32")
    assert rel_p(out[False][0], op) <= TOL["f32"] and rel_g(out[False][1], og) <= TOL["f32"]


def test_borrowed_context_rejects_a_short_workspace(pkg):
    import ctypes
    import torch
    I, J, K = 20, 12, 9
    L = pkg.lib()
    bufs = [torch.empty(pkg.field_bytes(I, J, K, "f32", 0), dtype=torch.uint8, device="cuda") for _ in range(2)]
    bufs += [torch.empty(pkg.field_bytes(I, J, K, "f32", q), dtype=torch.uint8, device="cuda") for q in range(1, 13)]
    g = pkg.jac_grid()
    g.I, g.J, g.K, g.prec, g.omega = I, J, K, 1, 0.8
    g.p[0], g.p[1] = bufs[0].data_ptr(), bufs[1].data_ptr()
    for q in range(1, 13):
        g.coef[q] = bufs[q + 1].data_ptr()
    need = pkg.ctx_workspace_size(I, J, K, "f32")
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    assert L.jac_create_borrowed(ctypes.byref(h), ctypes.byref(g), None, ctypes.c_void_p(ws.data_ptr()),
                                 ctypes.c_size_t(need - 256), None) == 1       # JAC_EINVAL
    assert b"workspace too small" in L.jac_last_error(None)
    assert L.jac_create_borrowed(ctypes.byref(h), ctypes.byref(g), None, ctypes.c_void_p(ws.data_ptr()),
                                 ctypes.c_size_t(need), None) == 0
    f = {k: torch.from_numpy(v).cuda() for k, v in ji.himeno_fields(I, J, K, seed=502).items()}
    fl = pkg.jac_fields()
    for q, name in enumerate(pkg.FIELDS):
        fl.f[q] = f[name].data_ptr()
    assert L.jac_upload_dev(h, ctypes.byref(fl)) == 0
    # a tape, or asynchronous staging, the workspace has no room for: JAC_ENOMEM, nothing allocated
    assert L.jac_tape_begin(h, 2, 4) == 2
    assert b"jac_set_workspace" in L.jac_last_error(h)
    assert L.jac_upload_async(h, ctypes.byref(fl)) == 2
    assert L.jac_destroy(h) == 0
