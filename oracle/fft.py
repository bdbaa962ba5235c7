"""FP64 CPU oracle of the 3-D complex FFT and the spectral step (ctypes wrapper
of fft_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this module.  The GPU
product path never imports it, and the two share no code.

What each function follows (the paper's second workload is NAS.FT, an FFT
application, Section 5.1.1; Section 6 names FFT function blocks as the next
offload target):
  * ``dft_axis``: the plain DFT of every line along one axis,
    X[k] = sum_j x[j] exp(sign 2 pi i j k / n), one O(n) sum per output.
  * ``fft3``: the axis DFTs along x, y, z (the separable definition of the
    3-D DFT); the inverse (sign = +1) is scaled by 1 / (n1 n2 n3).
  * ``evolve``: the exact Fourier-space solution of the heat equation on the
    periodic unit cube, inverse(U * exp(-4 pi^2 alpha t |kbar|^2)), and the
    energy sum |u|^2 of the result.
  * ``point``: one output of the 3-D DFT as a single sum over all points.

Arrays are complex128 numpy arrays of shape (n3, n2, n1) (x fastest).

Pins: tests/test_fft_oracle_pins.py checks this oracle against a delta, a
single Fourier mode, Parseval's identity, the inverse round trip, linearity,
the shift theorem, Hermitian symmetry of real input, the direct triple-sum
3-D DFT on tiny grids, numpy.fft, and the closed-form decay of a single mode
under the spectral step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fft_oracle.c")
_LIB = os.path.join(_HERE, "libfft_oracle.so")
_dp = ctypes.POINTER(ctypes.c_double)
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libfft_oracle.so with gcc (FP64, no FMA contraction, OpenMP)."""
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
            lib.fft_oracle_dft_axis.argtypes = [ctypes.c_int] * 5 + [_dp, _dp]
            lib.fft_oracle_fft3.argtypes = [ctypes.c_int] * 4 + [_dp, _dp]
            lib.fft_oracle_evolve.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 2 + [_dp, _dp, _dp]
            lib.fft_oracle_point.argtypes = [ctypes.c_int] * 4 + [_dp] + [ctypes.c_int] * 3 + [_dp]
            for fn in (lib.fft_oracle_dft_axis, lib.fft_oracle_fft3, lib.fft_oracle_evolve, lib.fft_oracle_point):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.ndim != 3:
        raise ValueError("expected a 3-D array of shape (n3, n2, n1)")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def dft_axis(x, axis: int, sign: int = -1) -> np.ndarray:
    """DFT of every line along ``axis`` (0: x = last numpy axis, 1: y, 2: z)."""
    a = _c128(x)
    n3, n2, n1 = a.shape
    out = np.empty_like(a)
    rc = _load().fft_oracle_dft_axis(n1, n2, n3, int(axis), int(sign), _ptr(a), _ptr(out))
    if rc:
        raise RuntimeError(f"fft_oracle_dft_axis failed ({rc})")
    return out


def fft3(x, sign: int = -1) -> np.ndarray:
    """3-D DFT (sign -1, unscaled) or its inverse (sign +1, scaled by 1/N)."""
    a = _c128(x)
    n3, n2, n1 = a.shape
    out = np.empty_like(a)
    rc = _load().fft_oracle_fft3(n1, n2, n3, int(sign), _ptr(a), _ptr(out))
    if rc:
        raise RuntimeError(f"fft_oracle_fft3 failed ({rc})")
    return out


def evolve(U, alpha: float, t: float):
    """(u(t), sum |u(t)|^2) for the forward transform U of the initial field."""
    a = _c128(U)
    n3, n2, n1 = a.shape
    out = np.empty_like(a)
    e = ctypes.c_double()
    rc = _load().fft_oracle_evolve(n1, n2, n3, float(alpha), float(t), _ptr(a), _ptr(out), ctypes.byref(e))
    if rc:
        raise RuntimeError(f"fft_oracle_evolve failed ({rc})")
    return out, e.value


def point(x, k, sign: int = -1) -> complex:
    """One output X[kx, ky, kz] (k = (kx, ky, kz)) of the unscaled 3-D DFT,
    from its definition as a single sum over all points (for sampled checks
    of grids too large for fft3)."""
    a = _c128(x)
    n3, n2, n1 = a.shape
    out = np.empty(2)
    rc = _load().fft_oracle_point(n1, n2, n3, int(sign), _ptr(a), int(k[0]), int(k[1]), int(k[2]), _ptr(out))
    if rc:
        raise RuntimeError(f"fft_oracle_point failed ({rc})")
    return complex(out[0], out[1])


__all__ = ["build", "dft_axis", "fft3", "evolve", "point"]
