"""Full-size adjoint on the 513 x 513 x 1025 grid (about 270 M points), through
the same context API and default plans the benchmark times, checked by
properties that hold at any size (the CPU oracle cannot hold the reverse pass
of this grid):

  * every sweep is affine in wrk1 and in the initial state p0, so the loss
    L = 1/2 |p_T - target|^2 is exactly quadratic in each, and for any
    direction d the central difference is exact:
        L(x + d) - L(x - d) = <dL/dx at x, (x + d) - (x - d)>;
    only rounding separates the two sides (FP64: 1e-11 of the difference,
    measured 2e-15 and 1e-13; FP32 storage, where the stored inputs and every
    state are rounded to FP32: 1e-5, measured 3e-8);
  * the recompute between checkpoints is deterministic, so the gradients do
    not depend on the checkpoint interval (bitwise);
  * faces carry no wrk1 or a3 gradient (the sweep never updates them)."""
import pytest

import jacobi_inputs as ji
from _util import OMEGA

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
I, J, K, T = 513, 513, 1025, 4
RTOL = {"f64": 1e-11, "f32": 1e-5}


@pytest.fixture(scope="module")
def problem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    fields = ji.himeno_fields_torch(I, J, K)
    target = torch.from_numpy(ji.target_field(I, J, K)).cuda()
    yield fields, target
    del fields, target
    torch.cuda.empty_cache()


def _stored(x, prec):
    """The values a precision stores for an FP64 input (FP32: RNE)."""
    return x if prec == "f64" else x.float().double()


def _loss(jac, fields, target):
    jac.upload_tensors(fields)
    jac.sweep(T)
    p = jac.download_tensor()
    return float(0.5 * ((p - target) ** 2).sum())


def _grads(jac, fields, target, C):
    jac.upload_tensors(fields)
    jac.tape_begin(C, T)
    jac.sweep(T)
    lam = jac.download_tensor() - target
    g = jac.sweep_adjoint(lam)
    jac.tape_end()
    return g


@pytest.mark.parametrize("prec,name", [("f32", "wrk1"), ("f64", "wrk1"), ("f64", "p")])
def test_exact_central_difference(problem, prec, name):
    import torch
    from paper_2002_12115_gb300 import Jacobi
    fields, target = problem
    # a smooth, one-signed direction, so that the difference of the losses
    # stands well above their rounding: 1e-3 (wrk1) or 1e-4 (p0) times a
    # positive sine bump over the whole grid
    k = torch.arange(K, dtype=torch.float64, device="cuda").view(K, 1, 1)
    j = torch.arange(J, dtype=torch.float64, device="cuda").view(1, J, 1)
    i = torch.arange(I, dtype=torch.float64, device="cuda").view(1, 1, I)
    bump = (0.5 + torch.sin(torch.pi * k / (K - 1)) * torch.sin(torch.pi * j / (J - 1))
            * torch.sin(torch.pi * i / (I - 1)))
    d = (1e-3 if name == "wrk1" else 1e-4) * bump
    del k, j, i, bump
    with Jacobi(I, J, K, prec, OMEGA) as jac:
        g = _grads(jac, fields, target, C=2)["g_p0" if name == "p" else "g_" + name]
        plus = dict(fields)
        plus[name] = fields[name] + d
        lp = _loss(jac, plus, target)
        minus = dict(fields)
        minus[name] = fields[name] - d
        d_eff = _stored(plus[name], prec) - _stored(minus[name], prec)
        del plus
        lm = _loss(jac, minus, target)
        del minus
    want = float((g * d_eff).sum())
    got = lp - lm
    err = abs(got - want) / abs(got)
    print(f"513x513x1025 {prec} d{name}: L+ - L- = {got:.9e}, <g, d> = {want:.9e}, rel {err:.2e}")
    assert err <= RTOL[prec], (got, want, err)


def test_checkpoint_interval_and_faces(problem):
    import torch
    from paper_2002_12115_gb300 import Jacobi
    fields, target = problem
    with Jacobi(I, J, K, "f32", OMEGA) as jac:
        g1 = _grads(jac, fields, target, C=1)
        g4 = _grads(jac, fields, target, C=4)
    for key in ("g_wrk1", "g_a3", "g_p0"):
        assert torch.equal(g1[key], g4[key]), key
    for key in ("g_wrk1", "g_a3"):
        gk = g1[key]
        faces = [gk[0], gk[-1], gk[:, 0], gk[:, -1], gk[:, :, 0], gk[:, :, -1]]
        assert all(int(torch.count_nonzero(f)) == 0 for f in faces), key
    assert float(g1["g_wrk1"].abs().max()) > 0


# ---------------------------------------------------------------------------
# The workload's own shape: 100 FP32 sweeps, the reverse pass over the last
# 20 with a checkpoint every 5 (what the benchmark times).
T_SWEEPS, T_TAPED, T_C = 100, 20, 5


@pytest.fixture(scope="module")
def config5_reverse(problem):
    """p_80 (FP64 copy of the FP32 state after 80 sweeps) and the gradients
    of L = 1/2 |p_100 - target|^2 with respect to the last 20 sweeps' wrk1,
    a3 and p_80, through the context API and default plans."""
    from paper_2002_12115_gb300 import Jacobi
    fields, target = problem
    with Jacobi(I, J, K, "f32", OMEGA) as jac:
        jac.upload_tensors(fields)
        jac.sweep(T_SWEEPS - T_TAPED)
        p80 = jac.download_tensor()
        jac.tape_begin(T_C, T_TAPED)
        jac.sweep(T_TAPED)
        lam = jac.download_tensor() - target
        g = jac.sweep_adjoint(lam)
    yield p80, g
    del p80, g


def _loss_from(jac, fields, target, p_start, n):
    f = dict(fields)
    f["p"] = p_start
    jac.upload_tensors(f)
    jac.sweep(n)
    p = jac.download_tensor()
    return float(0.5 * ((p - target) ** 2).sum())


@pytest.mark.parametrize("name", ["wrk1", "p"])
def test_config5_reverse_pass_exact_central_difference(problem, config5_reverse, name):
    """L over the last 20 sweeps, started from p_80, is exactly quadratic in
    wrk1 and in p_80: the central difference along a smooth direction equals
    <gradient, direction> up to FP32 storage rounding."""
    import torch
    from paper_2002_12115_gb300 import Jacobi
    fields, target = problem
    p80, g = config5_reverse
    k = torch.arange(K, dtype=torch.float64, device="cuda").view(K, 1, 1)
    j = torch.arange(J, dtype=torch.float64, device="cuda").view(1, J, 1)
    i = torch.arange(I, dtype=torch.float64, device="cuda").view(1, 1, I)
    bump = 0.5 + torch.sin(torch.pi * k / (K - 1)) * torch.sin(torch.pi * j / (J - 1)) * torch.sin(
        torch.pi * i / (I - 1))
    d = (1e-3 if name == "wrk1" else 1e-4) * bump
    del k, j, i, bump
    with Jacobi(I, J, K, "f32", OMEGA) as jac:
        if name == "wrk1":
            plus, minus = dict(fields), dict(fields)
            plus["wrk1"] = fields["wrk1"] + d
            minus["wrk1"] = fields["wrk1"] - d
            lp = _loss_from(jac, plus, target, p80, T_TAPED)
            lm = _loss_from(jac, minus, target, p80, T_TAPED)
            d_eff = _stored(plus["wrk1"], "f32") - _stored(minus["wrk1"], "f32")
            gk = g["g_wrk1"]
        else:
            lp = _loss_from(jac, fields, target, p80 + d, T_TAPED)
            lm = _loss_from(jac, fields, target, p80 - d, T_TAPED)
            d_eff = _stored(p80 + d, "f32") - _stored(p80 - d, "f32")
            gk = g["g_p0"]
    want = float((gk * d_eff).sum())
    got = lp - lm
    err = abs(got - want) / abs(got)
    print(f"513x513x1025 reverse pass of sweeps 81-100, C = 5, d{name}: {got:.9e} vs {want:.9e}, rel {err:.2e}")
    assert err <= RTOL["f32"], (got, want, err)


def test_config5_reverse_pass_gradients_against_oracle(problem, config5_reverse):
    """dL/dwrk1 and dL/da3 at 64 seeded interior points each (the
    finite-difference points of the workload), against the FP64 reverse-mode
    oracle run on the box of radius 42 around each point, from the same p_80
    and the FP32-rounded inputs.  A point's gradient depends only on the
    states within 19 points of it over the 20 sweeps, and the box's held
    faces reach at most 20 points in, so the box reproduces it.  Bar: 1e-4
    of the largest gradient sampled (FP32 state and adjoint against FP64)."""
    import numpy as np

    import oracle
    fields, target = problem
    p80, g = config5_reverse
    R = 42
    w_pts, a_pts = ji.fd_points(I, J, K, 64)
    got = {"g_wrk1": [], "g_a3": []}
    want = {"g_wrk1": [], "g_a3": []}
    for key, pts in (("g_wrk1", w_pts), ("g_a3", a_pts)):
        gk = g[key]
        for (i, j, k) in pts:
            lo = (max(0, i - R), max(0, j - R), max(0, k - R))
            hi = (min(I, i + R + 1), min(J, j + R + 1), min(K, k + R + 1))
            box = oracle.round_inputs(ji.himeno_fields_box(I, J, K, lo, hi), "f32")
            p0 = p80[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].cpu().numpy()
            tg = ji.target_field_box(I, J, K, lo, hi)
            r = oracle.adjoint(box, T_TAPED, tg, OMEGA, p0=p0)
            want[key].append(r[key][k - lo[2], j - lo[1], i - lo[0]])
            got[key].append(float(gk[k, j, i]))
    for key in got:
        a, b = np.array(got[key]), np.array(want[key])
        err = float(np.abs(a - b).max() / np.abs(b).max())
        print(f"513x513x1025 {key} at 64 points vs reverse-mode oracle: {err:.2e}")
        assert err <= 1e-4, (key, err)
