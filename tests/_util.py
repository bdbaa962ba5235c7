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
