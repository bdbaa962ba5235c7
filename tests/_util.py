"""Helpers shared by the GPU parity tests (GPU side through the C ABI, the
oracle side through oracle/; the two never share arithmetic)."""
import numpy as np

OMEGA = 0.8
TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 3e-3}


def gpu_run(fields, n, prec, plan=None, omega=OMEGA):
    from paper_2002_12115_gb300 import Jacobi
    K, J, I = fields["p"].shape
    with Jacobi(I, J, K, prec, omega) as jac:
        if plan is not None:
            jac.set_plan(*plan)
        jac.upload(fields)
        jac.sweep(n)
        g = jac.residual() if n > 0 else None
        return jac.download(), g


def oracle_ref(fields, n, prec, omega=OMEGA):
    """Oracle on the problem a precision stores: rounded inputs, and for the
    FP32-state paths the state rounded to FP32 after every sweep."""
    import oracle
    fr = oracle.round_inputs(fields, prec)
    return oracle.run(fr, n, omega, state="f64" if prec == "f64" else "f32")


def rel_p(p, q):
    return float(np.abs(p - q).max() / np.abs(q).max())


def rel_g(g, h):
    return abs(g - h) / abs(h) if h != 0 else abs(g)


def residual_ok(g, want, prec, n_int, pmax=1.0):
    """The residual bar: relative TOL, except on grids so small (n_int < 64)
    that a converged residual sits at the rounding level of the arithmetic.
    There every ss carries an absolute rounding error up to about
    delta = 16 eps |p|max, so the bar is the worst case of that error,
    sum(2 |ss| delta + delta^2) <= 2 sqrt(n_int gosa) delta + n_int delta^2
    (the state, which carries the real information, is still checked at TOL)."""
    if rel_g(g, want) <= TOL[prec]:
        return True
    eps = 2.0 ** -53 if prec == "f64" else 2.0 ** -24
    delta = 16 * eps * pmax
    return n_int < 64 and abs(g - want) <= 2 * np.sqrt(n_int * abs(want)) * delta + n_int * delta ** 2
