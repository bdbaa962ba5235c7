"""One adjoint sweep through the stateless C-ABI entry point
(jac_adjoint_step_dev) against the FP64 reverse-mode CPU oracle (scatter
form) for one sweep: lambda_t at every point, faces included (the output
starts as NaN, so a point left unwritten fails), and the FP64 gradient
accumulation (+=) on top of nonzero starting values.

Shapes cover one and several tiles in i, j and k, ragged last tiles, the
face column I-1 falling just past the last tile (I-1 a multiple of the tile
width, 64 points), a last row of tiles one row tall (FP32 tiles are 15 rows,
FP64 tiles 8), work items of one to a few output planes (both edge planes in
every item), and the smallest grids."""
import numpy as np
import pytest

import jacobi_inputs as ji

pytestmark = pytest.mark.gpu
OMEGA = 0.8
COEF = ("a0", "a1", "a2", "b0", "b1", "b2", "c0", "c1", "c2")
TOL = {"f64": 1e-13, "f32": 1e-5, "bf16": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    import oracle
    oracle.build()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def one_step(f, prec, target, kdepth=0, coef_grads=False, seed=0):
    """The GPU adjoint of one sweep from p0 for lambda_1 = p_1 - target, p_1
    the oracle's forward sweep.  Returns (got, want) dicts of dense arrays."""
    import torch

    import oracle
    from paper_2002_12115_gb300 import (Jacobi, adjoint_step_dev, pitch, stream_handle, unpack_dev, pack_dev,
                                        workspace_check, workspace_size)
    K, J, I = f["p"].shape
    fr = oracle.round_inputs(f, prec)
    want = oracle.adjoint(fr, 1, target, OMEGA, coef_grads=coef_grads)
    rng = np.random.default_rng(seed)
    # starting values of each gradient's own magnitude, so that taking them
    # off again costs no more than the rounding of the gradient itself
    g0 = {k: rng.uniform(-1, 1, (K, J, I)) * (np.abs(want[k]).max() if k in want else 1.0)
          for k in ("g_wrk1", "g_a3") + tuple("g_" + n for n in COEF)}
    st = stream_handle()
    dt = torch.float64 if prec == "f64" else torch.float32
    with Jacobi(I, J, K, prec, OMEGA) as jac:
        jac.upload(f)
        g = jac.grid()
        P = pitch(I)
        lam_dense = torch.from_numpy(np.ascontiguousarray(want["pT"] - target)).cuda()
        lam_in = torch.empty((K, J, P), dtype=dt, device="cuda")
        lam_out = torch.full((K, J, P), float("nan"), dtype=dt, device="cuda")
        pack_dev(I, J, K, prec, 0, lam_dense.data_ptr(), lam_in.data_ptr(), st)
        gd = {k: torch.from_numpy(v).cuda() for k, v in g0.items()}
        ws = torch.zeros(workspace_size(g), dtype=torch.uint8, device="cuda")
        gc = [gd["g_" + n].data_ptr() for n in COEF] if coef_grads else None
        adjoint_step_dev(g, g.p[0], lam_in.data_ptr(), lam_out.data_ptr(), gd["g_wrk1"].data_ptr(),
                         gd["g_a3"].data_ptr(), ws.data_ptr(), ws.numel(), st, g_coef=gc, kdepth=kdepth)
        workspace_check(ws.data_ptr(), st)
        out = torch.empty((K, J, I), dtype=torch.float64, device="cuda")
        unpack_dev(I, J, K, prec, 0, lam_out.data_ptr(), out.data_ptr(), st)
        torch.cuda.synchronize()
        got = {"g_p0": out.cpu().numpy()}
        for k, v in gd.items():
            got[k] = v.cpu().numpy() - g0[k]
    return got, want


CASES = [
    # prec, (I, J, K), kdepth
    ("f64", (3, 3, 3), 0), ("f64", (5, 6, 7), 1), ("f64", (65, 20, 13), 0), ("f64", (70, 13, 9), 3),
    ("f64", (129, 9, 11), 2),
    ("f32", (4, 4, 4), 1), ("f32", (33, 33, 65), 0), ("f32", (129, 17, 23), 0), ("f32", (130, 9, 11), 4),
    ("f32", (200, 19, 37), 7), ("f32", (257, 10, 6), 1),
    ("bf16", (129, 17, 23), 0), ("bf16", (257, 9, 12), 5), ("bf16", (50, 30, 20), 3),
    # FP32 tiles are 64 points x 15 rows: I - 1 a multiple of 64 (the face column is a
    # tile's extra column) and J one row past a multiple of 15 (a one-row last tile)
    ("f32", (65, 16, 9), 0), ("f32", (129, 31, 8), 2), ("bf16", (193, 46, 6), 0),
]


@pytest.mark.parametrize("prec,dims,kdepth", CASES)
def test_one_adjoint_sweep(prec, dims, kdepth):
    I, J, K = dims
    f = ji.himeno_fields(I, J, K, seed=500 + I + J + K)
    target = ji.target_field(I, J, K)
    got, want = one_step(f, prec, target, kdepth, seed=I)
    errs = {k: rel(got[k], want[k]) for k in ("g_p0", "g_wrk1", "g_a3")}
    assert all(np.isfinite(got[k]).all() for k in got), "a point of lambda_t was not written"
    assert all(v <= TOL[prec] for v in errs.values()), errs


@pytest.mark.parametrize("prec,dims,kdepth", [("f64", (65, 12, 10), 3), ("f32", (129, 11, 9), 2),
                                              ("bf16", (257, 9, 7), 0)])
def test_one_adjoint_sweep_coefficient_gradients(prec, dims, kdepth):
    I, J, K = dims
    f = ji.himeno_fields(I, J, K, seed=700 + I)
    target = ji.target_field(I, J, K)
    got, want = one_step(f, prec, target, kdepth, coef_grads=True, seed=K)
    for k in ("g_p0", "g_wrk1", "g_a3"):
        assert rel(got[k], want[k]) <= TOL[prec], (k, rel(got[k], want[k]))
    # A coefficient gradient is w times a state value or a bracket of four;
    # the bracket cancels, so its rounding is a few ulp of max|p|, not of
    # the bracket: elementwise bar 8 eps max|p| |w| on top of the relative
    # one (for one sweep g_wrk1 is w itself).
    eps = 2.0 ** -53 if prec == "f64" else 2.0 ** -24
    pmax = np.abs(oracle_round_p(f, prec)).max()
    for n in COEF:
        k = "g_" + n
        bar = TOL[prec] * np.abs(want[k]).max() + 8 * eps * pmax * np.abs(want["g_wrk1"])
        assert (np.abs(got[k] - want[k]) <= bar).all(), (k, rel(got[k], want[k]))


def oracle_round_p(f, prec):
    import oracle
    return oracle.round_inputs({"p": f["p"]}, prec)["p"] if prec != "f64" else f["p"]


def test_kdepth_does_not_change_the_result():
    """Every point's sum is formed in the same order whatever the item
    shape, so lambda_t and the gradients are bitwise the same."""
    I, J, K = 129, 19, 31
    f = ji.himeno_fields(I, J, K, seed=31)
    target = ji.target_field(I, J, K)
    ref, _ = one_step(f, "f32", target, 32)
    for kd in (1, 3, 8):
        got, _ = one_step(f, "f32", target, kd)
        for k in ("g_p0", "g_wrk1", "g_a3"):
            assert np.array_equal(got[k], ref[k]), (kd, k)


def test_entry_point_rejects_bad_arguments():
    import torch

    from paper_2002_12115_gb300 import JacError, Jacobi, adjoint_step_dev, stream_handle
    st = stream_handle()
    with Jacobi(9, 10, 11, "f32") as jac:
        jac.upload(ji.himeno_fields(9, 10, 11, seed=3))
        g = jac.grid()
        buf = torch.zeros(4096, dtype=torch.float32, device="cuda")
        ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
        ptr = buf.data_ptr()
        with pytest.raises(JacError, match="JAC_EINVAL"):      # lam_in == lam_out
            adjoint_step_dev(g, g.p[0], ptr, ptr, ptr, ptr, ws.data_ptr(), 256, st)
        with pytest.raises(JacError, match="JAC_EINVAL"):      # workspace too small
            adjoint_step_dev(g, g.p[0], ptr, ptr + 1024, ptr, ptr, ws.data_ptr(), 128, st)
        with pytest.raises(JacError, match="JAC_EINVAL"):      # misaligned lambda
            adjoint_step_dev(g, g.p[0], ptr + 4, ptr + 1024, ptr, ptr, ws.data_ptr(), 256, st)
        with pytest.raises(JacError, match="JAC_EINVAL"):      # negative kdepth
            adjoint_step_dev(g, g.p[0], ptr, ptr + 1024, ptr, ptr, ws.data_ptr(), 256, st, kdepth=-1)
