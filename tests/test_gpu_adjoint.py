"""GPU adjoint (transposed stencil, checkpointing, autograd) against the FP64
reverse-mode CPU oracle (scatter form) and central finite differences."""
import numpy as np
import pytest

import jacobi_inputs as ji

pytestmark = pytest.mark.gpu
OMEGA = 0.8
COEF = ("a0", "a1", "a2", "b0", "b1", "b2", "c0", "c1", "c2")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    import oracle
    oracle.build()


def _tensors(f):
    import torch
    t = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in f.items()}
    coefs = torch.stack([t[n] for n in COEF])
    return t, coefs


def gpu_grads(f, target, T, C, prec="f64", coef_grads=False):
    """L = 1/2 |p_T - target|^2 through torch autograd and libjac."""
    import torch
    from paper_2002_12115_gb300 import jacobi_sweep
    t, coefs = _tensors(f)
    p0 = t["p"].clone().requires_grad_(True)
    wrk1 = t["wrk1"].clone().requires_grad_(True)
    a3 = t["a3"].clone().requires_grad_(True)
    coefs = coefs.clone().requires_grad_(coef_grads)
    pT = jacobi_sweep(p0, wrk1, a3, coefs, t["bnd"], T, C, OMEGA, prec)
    tg = torch.from_numpy(target).cuda()
    loss = 0.5 * ((pT - tg) ** 2).sum()
    loss.backward()
    out = {"loss": float(loss.detach()), "pT": pT.detach().cpu().numpy(), "g_p0": p0.grad.cpu().numpy(),
           "g_wrk1": wrk1.grad.cpu().numpy(), "g_a3": a3.grad.cpu().numpy()}
    if coef_grads:
        for q, n in enumerate(COEF):
            out["g_" + n] = coefs.grad[q].cpu().numpy()
    return out


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("dims,T,C", [((3, 3, 3), 2, 1), ((4, 4, 4), 3, 2), ((5, 6, 7), 4, 4),
                                      ((40, 9, 11), 5, 2), ((70, 13, 9), 6, 4)])
def test_small_grids_all_gradients_fp64(dims, T, C):
    import oracle
    I, J, K = dims
    f = ji.himeno_fields(I, J, K, seed=300 + I)
    target = ji.target_field(I, J, K)
    want = oracle.adjoint(f, T, target, OMEGA, coef_grads=True)
    got = gpu_grads(f, target, T, C, "f64", coef_grads=True)
    assert rel(got["pT"], want["pT"]) <= 1e-13
    assert abs(got["loss"] - want["loss"]) <= 1e-12 * want["loss"]
    for k in ("g_p0", "g_wrk1", "g_a3") + tuple("g_" + n for n in COEF):
        assert rel(got[k], want[k]) <= 1e-12, (k, rel(got[k], want[k]))


@pytest.mark.slow
def test_config3_against_reverse_mode_oracle():
    """65 x 65 x 129, T = 50 FP64 sweeps, checkpoint every 10: gradients
    w.r.t. wrk1, a3 and p0 within 1e-10 (normwise) of the FP64 oracle."""
    import oracle
    I, J, K, T, C = 65, 65, 129, 50, 10
    f = ji.himeno_fields(I, J, K)
    target = ji.target_field(I, J, K)
    want = oracle.adjoint(f, T, target, OMEGA)
    got = gpu_grads(f, target, T, C, "f64")
    errs = {k: rel(got[k], want[k]) for k in ("g_p0", "g_wrk1", "g_a3")}
    print("config3 adjoint errors vs oracle:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(v <= 1e-10 for v in errs.values()), errs


@pytest.mark.slow
def test_config3_central_differences():
    """Central differences (h = 1e-6) of the GPU FP64 forward at 64 seeded
    entries each of wrk1 and a3.  L is quadratic in wrk1, so that check is
    exact up to rounding; the bar allows the central difference's rounding
    (about eps L / h) on top of 1e-6 max|g| + 1e-5 |g|."""
    import torch
    from paper_2002_12115_gb300 import Jacobi
    I, J, K, T, C = 65, 65, 129, 50, 10
    f = ji.himeno_fields(I, J, K)
    target = ji.target_field(I, J, K)
    got = gpu_grads(f, target, T, C, "f64")
    t, _ = _tensors(f)
    tg = torch.from_numpy(target).cuda()
    h = 1e-6
    jac = Jacobi(I, J, K, "f64", OMEGA)

    def loss(fields):
        jac.upload_tensors(fields)
        jac.sweep(T)
        p = jac.download_tensor()
        return float(0.5 * ((p - tg) ** 2).sum())

    pw, pa = ji.fd_points(I, J, K, 64)
    for name, pts in (("wrk1", pw), ("a3", pa)):
        g = got["g_" + name]
        for (i, j, k) in pts:
            base = t[name][k, j, i].item()
            fp = dict(t); fp[name] = t[name].clone(); fp[name][k, j, i] = base + h
            fm = dict(t); fm[name] = t[name].clone(); fm[name][k, j, i] = base - h
            fd = (loss(fp) - loss(fm)) / (2 * h)
            tol = 16 * np.finfo(float).eps * got["loss"] / h + 1e-6 * np.abs(g).max() + 1e-5 * abs(fd)
            assert abs(fd - g[k, j, i]) <= tol, (name, i, j, k, fd, g[k, j, i])
    jac.close()


def test_checkpoint_interval_does_not_change_gradients():
    """The recompute is deterministic, so the gradients are bitwise the same
    for every checkpoint interval."""
    I, J, K, T = 37, 21, 19, 12
    f = ji.himeno_fields(I, J, K, seed=9)
    target = ji.target_field(I, J, K)
    ref = gpu_grads(f, target, T, T, "f64")
    for C in (1, 5, 7):
        g = gpu_grads(f, target, T, C, "f64")
        for k in ("g_p0", "g_wrk1", "g_a3"):
            assert np.array_equal(g[k], ref[k]), (C, k)


@pytest.mark.parametrize("prec,tol", [("f32", 1e-4), ("bf16", 1e-3)])
def test_reduced_precision_adjoint(prec, tol):
    """FP32 / BF16-coefficient adjoints against the FP64 oracle run on the
    same rounded inputs; the gap is the FP32 rounding of state and lambda."""
    import oracle
    I, J, K, T, C = 41, 23, 29, 10, 5
    f = ji.himeno_fields(I, J, K, seed=12)
    target = ji.target_field(I, J, K)
    want = oracle.adjoint(oracle.round_inputs(f, prec), T, target, OMEGA)
    got = gpu_grads(f, target, T, C, prec)
    errs = {k: rel(got[k], want[k]) for k in ("g_p0", "g_wrk1", "g_a3")}
    print(f"{prec} adjoint errors vs oracle:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(v <= tol for v in errs.values()), errs


def test_tape_api_errors_and_state():
    import torch
    from paper_2002_12115_gb300 import JacError, Jacobi
    f = ji.himeno_fields(9, 10, 11, seed=1)
    t, _ = _tensors(f)
    with Jacobi(9, 10, 11, "f64") as jac:
        jac.upload_tensors(t)
        with pytest.raises(JacError, match="JAC_ESTATE"):
            jac.sweep_adjoint(torch.zeros_like(t["p"]))
        jac.sweep(3)
        g_before = jac.residual()
        jac.tape_begin(2, 4)
        jac.sweep(4)
        assert jac.tape_count() == 4
        with pytest.raises(JacError, match="JAC_ESTATE"):
            jac.sweep(1)                      # beyond the tape's size
        p = jac.download_tensor()
        r = jac.residual()
        jac.sweep_adjoint(torch.ones_like(p))
        assert torch.equal(jac.download_tensor(), p) and jac.residual() == r and r != g_before


@pytest.mark.parametrize("C", [3, 5, 6])
def test_two_sweep_recompute_gives_the_same_gradients(C):
    """Where the plan takes two-sweep passes (fuse = 2), the reverse pass
    recomputes a segment's states two per pass, storing the intermediate one;
    the states are bitwise those of single sweeps, so the gradients are
    bitwise those of a single-sweep recompute (fuse = 1), and they match the
    reverse-mode oracle.  Segments of 3, 5 and 6 sweeps leave 0 or 1 state to
    recompute singly; 17 taped sweeps leave a shorter last segment."""
    import torch
    import oracle
    from paper_2002_12115_gb300 import Jacobi
    I, J, K, T = 131, 20, 23, 17
    f = ji.himeno_fields(I, J, K, seed=21)
    target = ji.target_field(I, J, K)
    t, _ = _tensors(f)
    out = {}
    for fuse in (1, 2):
        with Jacobi(I, J, K, "f32") as jac:
            jac.set_plan(0, 0, 0, fuse)
            jac.upload_tensors(t)
            jac.tape_begin(C, T)
            jac.sweep(T)
            pT = jac.download_tensor()
            lam = pT - torch.from_numpy(target).cuda()
            g = jac.sweep_adjoint(lam)
            out[fuse] = {k: v.cpu().numpy() for k, v in g.items()}
    for k in ("g_p0", "g_wrk1", "g_a3"):
        assert np.array_equal(out[1][k], out[2][k]), k
    want = oracle.adjoint(oracle.round_inputs(f, "f32"), T, target, OMEGA)
    errs = {k: rel(out[2][k], want[k]) for k in ("g_p0", "g_wrk1", "g_a3")}
    assert all(v <= 1e-4 for v in errs.values()), errs
