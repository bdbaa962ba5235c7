"""FP64 CPU oracle of the 19-point Jacobi sweep (ctypes wrapper of jacobi_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this package.  The GPU
product path (``paper_2002_12115_gb300``) never imports it, and the two share
no code: the only module both use is ``jacobi_inputs`` (random inputs).

What each function follows:
  * ``run`` / ``sweep``: the Himeno-style Jacobi relaxation (Section 5.1.1
    names the Himeno benchmark, a Poisson solve by Jacobi iteration); the
    stencil, sweep and residual definition are written out in the header of
    jacobi_oracle.c.
  * ``adjoint``: reverse mode over T sweeps for L = 1/2 |p_T - target|^2,
    scatter form, all states kept.
  * ``round_inputs``: the storage rounding that the FP32 and BF16 paths apply
    (RNE to FP32; BF16 as RNE of the FP32 value), so that those paths are
    compared with the oracle on the same rounded problem.
  * ``sample_after``: p_n at chosen points of a large grid, by running the
    oracle on the box of radius n around each point (the sweep reaches one
    point per step in every direction, so points at the centre are exact).

Pins: tests/test_oracle_pins.py checks this oracle against closed forms
(constant fixed point, sine-mode decay), the boundary-mask invariant,
hand-expanded updates on 3^3 and 4^3 grids, mirror and axis-swap symmetry,
the single-sweep wrk1 derivative, finite differences and the adjoint
dot-product identity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FIELD_ORDER = ("a0", "a1", "a2", "a3", "b0", "b1", "b2", "c0", "c1", "c2", "wrk1", "bnd")
GRAD_COEF_ORDER = ("a0", "a1", "a2", "b0", "b1", "b2", "c0", "c1", "c2")

_dp = ctypes.POINTER(ctypes.c_double)


class _Fields(ctypes.Structure):
    _fields_ = [(n, _dp) for n in FIELD_ORDER]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, no FMA contraction, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = ctypes.c_int
            lib.oracle_sweep.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(_Fields), ctypes.c_double,
                                                              _dp, _dp, _dp, ctypes.c_int]
            lib.oracle_run.argtypes = [ctypes.c_int] * 3 + [ctypes.POINTER(_Fields), ctypes.c_double,
                                                            ctypes.c_int, _dp, _dp, ctypes.c_int]
            lib.oracle_adjoint.argtypes = ([ctypes.c_int] * 3 + [ctypes.POINTER(_Fields), ctypes.c_double,
                                                                 ctypes.c_int] + [_dp] * 8)
            for fn in (lib.oracle_sweep, lib.oracle_run, lib.oracle_adjoint):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 keeps it); returns the count in use."""
    return int(_load().oracle_set_threads(int(n)))


def _f64(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _pack(fields: dict):
    arrs = {n: _f64(fields[n]) for n in FIELD_ORDER}
    st = _Fields(*[_ptr(arrs[n]) for n in FIELD_ORDER])
    return st, arrs


def _dims(fields: dict):
    K, J, I = np.shape(fields["a0"])
    return int(I), int(J), int(K)


def sweep(fields: dict, p_in: np.ndarray, omega: float = 0.8, state: str = "f64"):
    """One sweep: returns (p_out, gosa).  state='f32' rounds the new state to FP32."""
    I, J, K = _dims(fields)
    st, keep = _pack(fields)
    pin = _f64(p_in).copy()
    pout = np.empty_like(pin)
    g = ctypes.c_double()
    rc = _load().oracle_sweep(I, J, K, ctypes.byref(st), omega, _ptr(pin), _ptr(pout), ctypes.byref(g),
                               _state_flag(state))
    if rc:
        raise RuntimeError(f"oracle_sweep failed ({rc})")
    return pout, g.value


def _state_flag(state: str) -> int:
    if state not in ("f64", "f32"):
        raise ValueError(state)
    return 1 if state == "f32" else 0


def run(fields: dict, n: int, omega: float = 0.8, p0: np.ndarray | None = None, state: str = "f64"):
    """n sweeps from p0 (default fields['p']): returns (p_n, gosa of sweep n).

    state='f32' models a state stored in FP32 between sweeps (the FP32 and
    BF16-coefficient paths store p in FP32): each new value is rounded to
    FP32, the arithmetic stays FP64."""
    I, J, K = _dims(fields)
    st, keep = _pack(fields)
    p = _f64(fields["p"] if p0 is None else p0).copy()
    g = ctypes.c_double()
    rc = _load().oracle_run(I, J, K, ctypes.byref(st), omega, int(n), _ptr(p), ctypes.byref(g),
                             _state_flag(state))
    if rc:
        raise RuntimeError(f"oracle_run failed ({rc})")
    return p, g.value


def adjoint(fields: dict, T: int, target: np.ndarray, omega: float = 0.8,
            p0: np.ndarray | None = None, coef_grads: bool = False) -> dict:
    """Reverse-mode gradients of L = 1/2 sum (p_T - target)^2 after T sweeps."""
    I, J, K = _dims(fields)
    st, keep = _pack(fields)
    p0a = _f64(fields["p"] if p0 is None else p0)
    tg = _f64(target)
    shape = (K, J, I)
    out = {k: np.empty(shape) for k in ("pT", "g_p0", "g_wrk1", "g_a3")}
    gc = np.empty((9,) + shape) if coef_grads else None
    loss = ctypes.c_double()
    rc = _load().oracle_adjoint(I, J, K, ctypes.byref(st), omega, int(T), _ptr(p0a), _ptr(tg),
                                ctypes.byref(loss), _ptr(out["pT"]), _ptr(out["g_p0"]),
                                _ptr(out["g_wrk1"]), _ptr(out["g_a3"]),
                                _ptr(gc) if gc is not None else None)
    if rc:
        raise RuntimeError(f"oracle_adjoint failed ({rc})")
    out["loss"] = loss.value
    if gc is not None:
        for q, name in enumerate(GRAD_COEF_ORDER):
            out["g_" + name] = gc[q]
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even of FP32 values to BF16, returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


STORAGE_COEFS = ("a0", "a1", "a2", "a3", "b0", "b1", "b2", "c0", "c1", "c2", "bnd")


def round_inputs(fields: dict, prec: str) -> dict:
    """The problem a storage precision actually solves, promoted back to FP64.

    prec 'f64': unchanged; 'f32': every array RNE to FP32; 'bf16': p and wrk1
    RNE to FP32, the eleven coefficient arrays (a*, b*, c*, bnd) RNE to FP32
    and then RNE to BF16.
    """
    if prec == "f64":
        return {k: _f64(v) for k, v in fields.items()}
    out = {}
    for k, v in fields.items():
        r = np.asarray(v, dtype=np.float32).astype(np.float64)
        if prec == "bf16" and k in STORAGE_COEFS:
            r = bf16_round(r)
        elif prec not in ("f32", "bf16"):
            raise ValueError(prec)
        out[k] = r
    return out


def sample_after(fields: dict, n: int, points, omega: float = 0.8, state: str = "f64"):
    """p_n at each (i, j, k) in ``points``, each from the oracle run on the
    sub-box of radius n around the point (clipped to the grid).  Points of the
    sub-box face that are not grid faces are held fixed, which is wrong for
    them but reaches the centre only after n + 1 sweeps."""
    I, J, K = _dims(fields)
    vals = []
    for (i, j, k) in points:
        lo = [max(0, c - n) for c in (k, j, i)]
        hi = [min(d - 1, c + n) + 1 for c, d in zip((k, j, i), (K, J, I))]
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        sub = {name: np.ascontiguousarray(v[sl]) for name, v in fields.items()}
        p, _ = run(sub, n, omega, state=state)
        vals.append(p[k - lo[0], j - lo[1], i - lo[2]])
    return np.asarray(vals)


__all__ = ["build", "set_threads", "sweep", "run", "adjoint", "round_inputs", "bf16_round",
           "sample_after", "FIELD_ORDER", "GRAD_COEF_ORDER"]

if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
