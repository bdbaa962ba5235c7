"""Seeded synthetic inputs for the 19-point variable-coefficient Jacobi sweep.

This module is shared by the CPU oracle (``oracle/``), the tests and the
benchmark.  It holds random-number generation and the input recipes only; it
contains none of the sweep's arithmetic (no stencil, no residual, no rounding
to a storage precision).

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), in its usual 64-bit form: the n-th output
(n = 1, 2, ...) of a stream seeded with ``s`` is ``mix(s + n * GAMMA)`` with
GAMMA = 0x9E3779B97F4A7C15 and ``mix`` the two xor-shift-multiply rounds.
Being counter based, any stretch of a stream can be produced independently,
which lets large arrays be generated in parallel chunks.

Uniform draws: ``U[lo, hi) = lo + (hi - lo) * (top 53 bits / 2**53)``.

Recipe of one grid (the Himeno-style workload of Section 5.1.1, whose sizes
the paper does not state; shapes follow the usual 2^n+1 grid sizes):
  * draws, in this order, N = I*J*K values each, i fastest, then j, then k:
    a0, a1, a2 ~ U[0.95, 1.05); b0, b1, b2 ~ U[-0.02, 0.02);
    c0, c1, c2 ~ U[0.95, 1.05); wrk1 ~ U[-1e-3, 1e-3); p-noise ~ U[-1e-3, 1e-3)
  * a3 = 1 / (a0 + a1 + a2 + c0 + c1 + c2), summed left to right in FP64
  * p0 = (k / (K-1))**2 + p-noise, at every point, faces included
  * bnd = 1 on the interior, 0 on the six faces
All arrays are float64 with shape (K, J, I), C-contiguous, so the flat index
of (i, j, k) is (k*J + j)*I + i.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

#: seed of grid 0 (a batch's grid g uses SEED + g)
SEED = 42
#: seed of the stream that draws the batch grid dimensions
BATCH_DIMS_SEED = 42 + 1_000_003
#: seed of the adjoint's target field
TARGET_SEED = 43
#: seed of the finite-difference sample positions
FD_SEED = 44
#: seed of sampled check positions on large grids
SAMPLE_SEED = 45
#: seed of the complex fields of the 3-D FFT workload
FFT_SEED = 46
#: grid sizes the batched workload draws from
BATCH_DIM_CHOICES = (17, 33, 49, 65, 97, 129)

COEF_NAMES = ("a0", "a1", "a2", "b0", "b1", "b2", "c0", "c1", "c2")
#: the eleven drawn arrays, in draw order
DRAW_ORDER = COEF_NAMES + ("wrk1", "pnoise")
#: every array of one grid, in the order the C-ABI field structs list them
FIELD_NAMES = ("p", "a0", "a1", "a2", "a3", "b0", "b1", "b2", "c0", "c1", "c2", "wrk1", "bnd")

_CHUNK = 1 << 22


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start+1 .. start+count (1-based) of the stream seeded with ``seed``."""
    with np.errstate(over="ignore"):
        n = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + n * GAMMA
        return _mix(z)


def splitmix64_scalar(seed: int, n: int) -> int:
    """The n-th output (1-based) of the stream, in plain Python integers."""
    z = (seed + n * 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def _unit(z: np.ndarray) -> np.ndarray:
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, start: int, count: int, lo: float, hi: float,
            out: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """U[lo, hi) draws start+1 .. start+count of the stream, in parallel chunks."""
    if out is None:
        out = np.empty(count, dtype=np.float64)
    span = hi - lo

    def work(c0: int) -> None:
        c1 = min(count, c0 + _CHUNK)
        u = _unit(splitmix64(seed, start + c0, c1 - c0))
        out[c0:c1] = lo + span * u

    starts = range(0, count, _CHUNK)
    if count <= _CHUNK:
        for c in starts:
            work(c)
    else:
        nt = threads or min(32, os.cpu_count() or 1)
        with ThreadPoolExecutor(nt) as ex:
            list(ex.map(work, starts))
    return out


_RANGES = {
    "a0": (0.95, 1.05), "a1": (0.95, 1.05), "a2": (0.95, 1.05),
    "b0": (-0.02, 0.02), "b1": (-0.02, 0.02), "b2": (-0.02, 0.02),
    "c0": (0.95, 1.05), "c1": (0.95, 1.05), "c2": (0.95, 1.05),
    "wrk1": (-1e-3, 1e-3), "pnoise": (-1e-3, 1e-3),
}


def interior_mask(I: int, J: int, K: int) -> np.ndarray:
    """1.0 on interior points, 0.0 on the six faces; shape (K, J, I)."""
    m = np.zeros((K, J, I), dtype=np.float64)
    m[1:K - 1, 1:J - 1, 1:I - 1] = 1.0
    return m


def himeno_fields(I: int, J: int, K: int, seed: int = SEED) -> dict[str, np.ndarray]:
    """All thirteen arrays of one grid, as described in the module docstring."""
    if min(I, J, K) < 3:
        raise ValueError("every grid dimension must be at least 3")
    N = I * J * K
    f: dict[str, np.ndarray] = {}
    for q, name in enumerate(DRAW_ORDER):
        lo, hi = _RANGES[name]
        f[name] = uniform(seed, q * N, N, lo, hi).reshape(K, J, I)
    s = f["a0"] + f["a1"]
    s += f["a2"]
    s += f["c0"]
    s += f["c1"]
    s += f["c2"]
    f["a3"] = np.reciprocal(s, out=s)
    kk = np.arange(K, dtype=np.float64) / float(K - 1)
    noise = f.pop("pnoise")
    noise += (kk * kk)[:, None, None]
    f["p"] = noise
    f["bnd"] = interior_mask(I, J, K)
    return {name: f[name] for name in FIELD_NAMES}


def himeno_fields_box(I: int, J: int, K: int, lo, hi, seed: int = SEED) -> dict[str, np.ndarray]:
    """The arrays of himeno_fields(I, J, K) restricted to the box
    lo <= (i, j, k) < hi, drawn directly: the generator is counter based, so
    each row of the box is the stretch of draws at its flat indices.  Equal,
    bitwise, to slicing the full arrays (tested); for sampled checks of grids
    too large to generate whole on the host."""
    (i0, j0, k0), (i1, j1, k1) = lo, hi
    if not (0 <= i0 < i1 <= I and 0 <= j0 < j1 <= J and 0 <= k0 < k1 <= K):
        raise ValueError("box outside the grid")
    N = I * J * K
    ni, nj, nk = i1 - i0, j1 - j0, k1 - k0
    flat = ((np.arange(k0, k1, dtype=np.uint64)[:, None, None] * np.uint64(J)
             + np.arange(j0, j1, dtype=np.uint64)[None, :, None]) * np.uint64(I)
            + np.arange(i0, i1, dtype=np.uint64)[None, None, :])
    f: dict[str, np.ndarray] = {}
    with np.errstate(over="ignore"):
        for q, name in enumerate(DRAW_ORDER):
            lo_v, hi_v = _RANGES[name]
            n = flat + np.uint64(q * N + 1)          # 1-based draw numbers of the box's points
            z = np.uint64(seed & _MASK64) + n * GAMMA
            f[name] = lo_v + (hi_v - lo_v) * _unit(_mix(z))
    s = f["a0"] + f["a1"]
    s += f["a2"]
    s += f["c0"]
    s += f["c1"]
    s += f["c2"]
    f["a3"] = np.reciprocal(s, out=s)
    kk = np.arange(k0, k1, dtype=np.float64) / float(K - 1)
    noise = f.pop("pnoise")
    noise += (kk * kk)[:, None, None]
    f["p"] = noise
    f["bnd"] = interior_mask(I, J, K)[k0:k1, j0:j1, i0:i1].copy() if N <= 1 << 22 else _box_mask(I, J, K, lo, hi)
    return {name: f[name] for name in FIELD_NAMES}


def _box_mask(I, J, K, lo, hi):
    """interior_mask(I, J, K) on the box lo <= (i, j, k) < hi, without the full array."""
    i = np.arange(lo[0], hi[0])
    j = np.arange(lo[1], hi[1])
    k = np.arange(lo[2], hi[2])
    mi = ((i >= 1) & (i <= I - 2)).astype(np.float64)
    mj = ((j >= 1) & (j <= J - 2)).astype(np.float64)
    mk = ((k >= 1) & (k <= K - 2)).astype(np.float64)
    return mk[:, None, None] * mj[None, :, None] * mi[None, None, :]


def target_field_box(I: int, J: int, K: int, lo, hi, seed: int = TARGET_SEED) -> np.ndarray:
    """target_field(I, J, K) restricted to the box lo <= (i, j, k) < hi."""
    out = np.zeros((hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]), dtype=np.float64)
    ii = np.arange(lo[0], hi[0], dtype=np.float64)
    jj = np.arange(lo[1], hi[1], dtype=np.float64)
    kk = np.arange(lo[2], hi[2], dtype=np.float64)
    for l, m, n in target_modes(seed):
        si = np.sin(np.pi * l * ii / (I - 1))
        sj = np.sin(np.pi * m * jj / (J - 1))
        sk = np.sin(np.pi * n * kk / (K - 1))
        out += 0.1 * sk[:, None, None] * sj[None, :, None] * si[None, None, :]
    return out


def batch_dims(n_grids: int, seed: int = BATCH_DIMS_SEED) -> list[tuple[int, int, int]]:
    """(I, J, K) of each batch grid: three draws per grid, each picks one of
    BATCH_DIM_CHOICES uniformly as floor(6u)."""
    u = _unit(splitmix64(seed, 0, 3 * n_grids))
    idx = np.minimum((u * len(BATCH_DIM_CHOICES)).astype(np.int64), len(BATCH_DIM_CHOICES) - 1)
    ch = np.asarray(BATCH_DIM_CHOICES)[idx].reshape(n_grids, 3)
    return [tuple(int(x) for x in row) for row in ch]


def target_modes(seed: int = TARGET_SEED) -> list[tuple[int, int, int]]:
    """Three (l, m, n) mode numbers in {1, 2, 3}, drawn l1, m1, n1, l2, ... as 1 + floor(3u)."""
    u = _unit(splitmix64(seed, 0, 9))
    v = 1 + np.minimum((u * 3).astype(np.int64), 2)
    return [tuple(int(x) for x in v[3 * m:3 * m + 3]) for m in range(3)]


def target_field(I: int, J: int, K: int, seed: int = TARGET_SEED) -> np.ndarray:
    """Smooth target of the adjoint loss: a sum of three sine modes, amplitude 0.1."""
    out = np.zeros((K, J, I), dtype=np.float64)
    ii = np.arange(I, dtype=np.float64)
    jj = np.arange(J, dtype=np.float64)
    kk = np.arange(K, dtype=np.float64)
    for l, m, n in target_modes(seed):
        si = np.sin(np.pi * l * ii / (I - 1))
        sj = np.sin(np.pi * m * jj / (J - 1))
        sk = np.sin(np.pi * n * kk / (K - 1))
        out += 0.1 * sk[:, None, None] * sj[None, :, None] * si[None, None, :]
    return out


def interior_points(I: int, J: int, K: int, count: int, seed: int, start: int = 0) -> np.ndarray:
    """``count`` interior (i, j, k) triples, each coordinate 1 + floor(u * (dim-2)),
    drawn i, j, k per point from draw ``start`` on; shape (count, 3)."""
    u = _unit(splitmix64(seed, start, 3 * count)).reshape(count, 3)
    dims = np.array([I - 2, J - 2, K - 2], dtype=np.float64)
    pts = 1 + np.minimum((u * dims).astype(np.int64), (dims - 1).astype(np.int64))
    return pts


def fd_points(I: int, J: int, K: int, count: int = 64) -> tuple[np.ndarray, np.ndarray]:
    """Positions for the finite-difference gradient checks: ``count`` interior
    points for wrk1, then ``count`` for a3, from the stream seeded with FD_SEED."""
    pts = interior_points(I, J, K, 2 * count, FD_SEED)
    return pts[:count], pts[count:]


# ------------------------------------------------------------------ torch
# The same recipe with torch tensors (for example on the GPU, where large
# workloads are generated in seconds).  SplitMix64 is evaluated in int64
# two's-complement arithmetic: products wrap modulo 2^64 exactly as for
# uint64, and the logical right shifts are arithmetic shifts with the sign
# bits masked off.  Bit-identical to the numpy version (tested).
def _as_i64(u: int) -> int:
    u &= _MASK64
    return u - (1 << 64) if u >= (1 << 63) else u


def _torch_mix(z):
    import torch
    z = (z ^ ((z >> 30) & ((1 << 34) - 1))) * _as_i64(0xBF58476D1CE4E5B9)
    z = (z ^ ((z >> 27) & ((1 << 37) - 1))) * _as_i64(0x94D049BB133111EB)
    return z ^ ((z >> 31) & ((1 << 33) - 1))


def uniform_torch(seed: int, start: int, count: int, lo: float, hi: float, device="cuda", chunk: int = 1 << 26):
    """U[lo, hi) draws start+1 .. start+count as a float64 torch tensor."""
    import torch
    out = torch.empty(count, dtype=torch.float64, device=device)
    g = _as_i64(0x9E3779B97F4A7C15)
    s = _as_i64(seed)
    for c0 in range(0, count, chunk):
        c1 = min(count, c0 + chunk)
        n = torch.arange(start + c0 + 1, start + c1 + 1, dtype=torch.int64, device=device)
        z = _torch_mix(n * g + s)
        u = ((z >> 11) & ((1 << 53) - 1)).to(torch.float64) * (1.0 / 9007199254740992.0)
        out[c0:c1] = lo + (hi - lo) * u
    return out


def himeno_fields_torch(I: int, J: int, K: int, seed: int = SEED, device="cuda") -> dict:
    """himeno_fields as float64 torch tensors of shape (K, J, I) on `device`."""
    import torch
    if min(I, J, K) < 3:
        raise ValueError("every grid dimension must be at least 3")
    N = I * J * K
    f = {}
    for q, name in enumerate(DRAW_ORDER):
        lo, hi = _RANGES[name]
        f[name] = uniform_torch(seed, q * N, N, lo, hi, device).view(K, J, I)
    s = f["a0"] + f["a1"]
    s += f["a2"]
    s += f["c0"]
    s += f["c1"]
    s += f["c2"]
    f["a3"] = torch.reciprocal(s)
    del s
    kk = torch.arange(K, dtype=torch.float64, device=device) / float(K - 1)
    p = f.pop("pnoise")
    p += (kk * kk).view(K, 1, 1)
    f["p"] = p
    bnd = torch.zeros((K, J, I), dtype=torch.float64, device=device)
    bnd[1:K - 1, 1:J - 1, 1:I - 1] = 1.0
    f["bnd"] = bnd
    return {name: f[name] for name in FIELD_NAMES}


# ------------------------------------------------------------------ FFT
# Inputs of the 3-D FFT workload (the paper's second application, NAS.FT, is
# an FFT code, Section 5.1.1).  A complex field of shape (n3, n2, n1), x
# fastest: real parts are draws 1 .. N of the stream, imaginary parts draws
# N+1 .. 2N, each U[-1, 1).
def fft_field(n1: int, n2: int, n3: int, seed: int = FFT_SEED) -> np.ndarray:
    """Seeded complex128 field of shape (n3, n2, n1)."""
    N = n1 * n2 * n3
    out = np.empty((n3, n2, n1), dtype=np.complex128)
    out.real = uniform(seed, 0, N, -1.0, 1.0).reshape(n3, n2, n1)
    out.imag = uniform(seed, N, N, -1.0, 1.0).reshape(n3, n2, n1)
    return out


def fft_field_torch(n1: int, n2: int, n3: int, seed: int = FFT_SEED, device="cuda"):
    """fft_field as a complex128 torch tensor on ``device`` (bitwise equal)."""
    import torch
    N = n1 * n2 * n3
    re = uniform_torch(seed, 0, N, -1.0, 1.0, device)
    im = uniform_torch(seed, N, N, -1.0, 1.0, device)
    return torch.complex(re, im).view(n3, n2, n1)
