"""torch.autograd bridge of the hand-written adjoint sweep.

``JacobiSweep.apply(p0, wrk1, a3, coefs, bnd, T, C, omega, prec)`` runs T
sweeps on the GPU (libjac) and returns p_T; its backward runs libjac's
reverse pass (checkpoint every C sweeps, recompute in between, transposed
stencil in gather form, FP64 gradient accumulation) and returns dL/dp0,
dL/dwrk1, dL/da3 and, when ``coefs`` requires grad, dL/d(a0..c2).

All tensors are float64 CUDA tensors of shape (K, J, I) (``coefs``: (9, K,
J, I) in the order a0, a1, a2, b0, b1, b2, c0, c1, c2); ``prec`` picks the
storage/arithmetic precision of the GPU path ("f64", "f32", "bf16").
"""
from __future__ import annotations

import torch

from .binding import Jacobi

COEF_ORDER = ("a0", "a1", "a2", "b0", "b1", "b2", "c0", "c1", "c2")


class JacobiSweep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p0, wrk1, a3, coefs, bnd, T: int, C: int, omega: float = 0.8, prec: str = "f64"):
        K, J, I = p0.shape
        for name, t in (("p0", p0), ("wrk1", wrk1), ("a3", a3), ("bnd", bnd)):
            if t.shape != p0.shape or t.dtype != torch.float64 or not t.is_cuda:
                raise ValueError(f"{name} must be a float64 CUDA tensor of shape {tuple(p0.shape)}")
        if coefs.shape != (9,) + tuple(p0.shape) or coefs.dtype != torch.float64:
            raise ValueError("coefs must be float64 of shape (9, K, J, I)")
        fields = {"p": p0.contiguous(), "a3": a3.contiguous(), "wrk1": wrk1.contiguous(),
                  "bnd": bnd.contiguous()}
        cc = coefs.contiguous()
        for q, name in enumerate(COEF_ORDER):
            fields[name] = cc[q]
        # a borrowed context: storage, staging and the tape are torch tensors
        # (the caching allocator), sized for this tape up front
        jac = Jacobi(I, J, K, prec, omega, tape=(C, T) if T > 0 else None)
        jac.upload_tensors(fields)
        if T > 0:
            jac.tape_begin(C, T)
            jac.sweep(T)
        pT = jac.download_tensor()
        ctx.jac = jac
        ctx.T = T
        ctx.shape = tuple(p0.shape)
        return pT

    @staticmethod
    def backward(ctx, g):
        jac = ctx.jac
        if jac is None:
            raise RuntimeError("JacobiSweep supports one backward pass per forward: its tape is released "
                               "after the first (retain_graph=True does not keep it)")
        need_p0, need_w, need_a3, need_c = ctx.needs_input_grad[:4]
        if ctx.T == 0:
            z = torch.zeros_like(g)
            out = (g if need_p0 else None, z if need_w else None, z if need_a3 else None,
                   torch.zeros((9,) + ctx.shape, dtype=g.dtype, device=g.device) if need_c else None)
        else:
            r = jac.sweep_adjoint(g.to(torch.float64).contiguous(), coef_grads=need_c, want_p0=need_p0)
            gc = torch.stack([r["g_" + n] for n in COEF_ORDER]) if need_c else None
            out = (r.get("g_p0"), r["g_wrk1"] if need_w else None, r["g_a3"] if need_a3 else None, gc)
        jac.close()
        ctx.jac = None
        return out + (None, None, None, None, None)


def jacobi_sweep(p0, wrk1, a3, coefs, bnd, T: int, C: int, omega: float = 0.8, prec: str = "f64"):
    """Differentiable T-sweep map (p0, wrk1, a3, coefs) -> p_T on the GPU."""
    return JacobiSweep.apply(p0, wrk1, a3, coefs, bnd, int(T), int(C), float(omega), prec)
