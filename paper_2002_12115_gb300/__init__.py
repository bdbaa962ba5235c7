"""GB300-native 19-point variable-coefficient Jacobi relaxation (libjac).

The hot path of the loop-nest applications that Yamato's automatic GPU
offloading targets (the Himeno benchmark of Section 5.1.1): a device-resident
3-D 19-point Jacobi sweep with a fused residual, behind the C ABI in
include/jacobi.h, with hand-written sm_103a CUDA kernels.

    from paper_2002_12115_gb300 import Jacobi
    with Jacobi(I, J, K, prec="f32") as jac:
        jac.upload(fields)        # one copy-in
        jac.sweep(1000)           # resident sweeps
        gosa = jac.residual()     # residual of the last sweep
        p = jac.download()        # one copy-out
"""
from .binding import (FFT3, FIELDS, KDEPTH_BALANCED, PRECS, JacError, Jacobi, JacobiBatch, adjoint_step_dev, check,
                      ctx_workspace_size, fft_workspace_size, field_bytes, jac_fields, jac_grid, jac_plan, jac_ws_spec, lib, pack_dev,
                      pitch, resolve_plan, stream_handle, sweep_dev, unpack_dev, workspace_check, workspace_size)


def __getattr__(name):
    # torch-dependent parts load lazily
    if name in ("JacobiSweep", "jacobi_sweep"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)


__all__ = ["FFT3", "FIELDS", "KDEPTH_BALANCED", "PRECS", "JacError", "Jacobi", "JacobiBatch", "JacobiSweep",
           "adjoint_step_dev", "check", "ctx_workspace_size", "fft_workspace_size", "field_bytes", "jac_fields", "jac_grid", "jac_plan",
           "jac_ws_spec", "jacobi_sweep", "lib", "pack_dev", "pitch", "resolve_plan", "stream_handle", "sweep_dev",
           "unpack_dev", "workspace_check", "workspace_size"]
