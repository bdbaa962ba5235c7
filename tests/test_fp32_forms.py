"""Why the FP32 path evaluates ss in difference form (a numerical probe on the
CPU, not the oracle and not the kernel).

Late in a run ss is small against p (|ss| ~ 1e-5 |p| on 129x129x257), so the
written form s0 * a3 - p cancels almost every bit of an FP32 s0 * a3.  The
difference form a3 * (sum_d coef_d (p_nb - p) + b-terms + wrk1) + p (a3 S - 1),
with S = a0 + a1 + a2 + c0 + c1 + c2, is the same number algebraically but
never forms the two large nearly equal terms.  This probe evaluates both forms
in FP32 (numpy float32, no fused multiply-add) on a late state and compares the
residual sum of squares with the FP64 definition."""
import numpy as np

import jacobi_inputs as ji

OMEGA = 0.8


def neighbours(p):
    """Views of p shifted to each of the 18 neighbours of the interior points."""
    c = p[1:-1, 1:-1, 1:-1]

    def at(dk, dj, di):
        K, J, I = p.shape
        return p[1 + dk:K - 1 + dk, 1 + dj:J - 1 + dj, 1 + di:I - 1 + di]
    return c, at


def ss_fp64(f, p):
    c, at = neighbours(p)
    g = {k: v[1:-1, 1:-1, 1:-1] for k, v in f.items()}
    s0 = (g["a0"] * at(0, 0, 1) + g["a1"] * at(0, 1, 0) + g["a2"] * at(1, 0, 0)
          + g["b0"] * (at(0, 1, 1) - at(0, -1, 1) - at(0, 1, -1) + at(0, -1, -1))
          + g["b1"] * (at(1, 1, 0) - at(-1, 1, 0) - at(1, -1, 0) + at(-1, -1, 0))
          + g["b2"] * (at(1, 0, 1) - at(-1, 0, 1) - at(1, 0, -1) + at(-1, 0, -1))
          + g["c0"] * at(0, 0, -1) + g["c1"] * at(0, -1, 0) + g["c2"] * at(-1, 0, 0) + g["wrk1"])
    return (s0 * g["a3"] - c) * g["bnd"]


def ss_fp32_written(f, p):
    f32 = {k: v.astype(np.float32) for k, v in f.items()}
    return ss_fp64(f32, p.astype(np.float32))


def ss_fp32_difference(f, p):
    p = p.astype(np.float32)
    g = {k: v[1:-1, 1:-1, 1:-1].astype(np.float32) for k, v in f.items()}
    c, at = neighbours(p)
    d = (g["wrk1"] + g["a0"] * (at(0, 0, 1) - c) + g["a1"] * (at(0, 1, 0) - c) + g["a2"] * (at(1, 0, 0) - c)
         + g["c0"] * (at(0, 0, -1) - c) + g["c1"] * (at(0, -1, 0) - c) + g["c2"] * (at(-1, 0, 0) - c)
         + g["b0"] * (at(0, 1, 1) - at(0, -1, 1) - at(0, 1, -1) + at(0, -1, -1))
         + g["b1"] * (at(1, 1, 0) - at(-1, 1, 0) - at(1, -1, 0) + at(-1, -1, 0))
         + g["b2"] * (at(1, 0, 1) - at(-1, 0, 1) - at(1, 0, -1) + at(-1, 0, -1)))
    # a3 S - 1 from the FP32 coefficients, with S summed exactly in FP64 (the
    # kernel sums it exactly in FP32 by compensation) and one rounding to FP32
    S = sum(g[k].astype(np.float64) for k in ("a0", "a1", "a2", "c0", "c1", "c2"))
    ec = (g["a3"].astype(np.float64) * S - 1.0).astype(np.float32)
    return (g["a3"] * d + c * ec) * g["bnd"]


def test_difference_form_keeps_the_fp32_residual():
    """On the state after 1000 sweeps of a 65x65x129 grid (FP32-rounded
    inputs, so both forms see the same problem; measured here: written form
    1.0e-5, difference form 1.3e-9) the difference form's residual agrees with
    the FP64 definition far inside the FP32 bar, and the written form's error
    is at least a hundred times larger, already at the bar.  It grows as ss
    shrinks against p: larger grids and later sweeps."""
    import oracle
    oracle.build()
    f = oracle.round_inputs(ji.himeno_fields(65, 65, 129), "f32")
    p, _ = oracle.run(f, 1000, OMEGA, state="f32")
    ref = float(np.sum(ss_fp64(f, p) ** 2))
    err_written = abs(float(np.sum(ss_fp32_written(f, p).astype(np.float64) ** 2)) - ref) / ref
    err_diff = abs(float(np.sum(ss_fp32_difference(f, p).astype(np.float64) ** 2)) - ref) / ref
    print(f"residual error, FP32 written form {err_written:.2e}, difference form {err_diff:.2e}")
    assert err_diff <= 1e-7
    assert err_written >= 100 * err_diff
