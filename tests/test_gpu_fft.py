"""The 3-D FFT block (include/jfft.h) against the FP64 FFT oracle.

Tolerances (normwise, max|dX| / max|X|): FP64 storage 1e-12; FP32 storage
1e-5.  A radix-2..16 FFT of length n rounds each output through log2(n)
butterfly levels and one twiddle product per stage, so its error grows like
eps * log2(N) (N = n1 n2 n3 over the three passes): about 6e-8 * 27 = 1.6e-6
for the largest grid here against max|X|, with room for the twiddle
table's own rounding.  FP32 inputs are rounded to complex64 before the
oracle sees them (the oracle transforms the same numbers).

Shapes cover every supported length 2 .. 1024 on each axis, ragged
combinations, in-place and out-of-place calls, and the spectral step with
its energy sum."""
import numpy as np
import pytest

import jacobi_inputs as ji

pytestmark = pytest.mark.gpu
TOL = {"c64": 1e-12, "c32": 1e-5}

SHAPES = [(2, 4, 8), (16, 2, 4), (4, 32, 2), (64, 8, 16), (128, 4, 2), (8, 128, 16), (32, 16, 128),
          (256, 8, 4), (4, 256, 8), (16, 4, 256), (512, 2, 4), (8, 512, 2), (2, 4, 512), (1024, 4, 2),
          (2, 1024, 4), (4, 2, 1024), (64, 64, 64)]


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_12115_gb300 import _build
    _build.build()
    import oracle.fft
    oracle.fft.build()
    import paper_2002_12115_gb300 as p
    return p


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _dev(x, prec):
    import torch
    t = torch.from_numpy(x)
    return (t.to(torch.complex64) if prec == "c32" else t).cuda()


@pytest.mark.parametrize("prec", ["c64", "c32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_forward_and_inverse_match_oracle(pkg, shape, prec):
    import oracle.fft as fo
    n1, n2, n3 = shape
    x = ji.fft_field(n1, n2, n3, seed=600 + n1 + 3 * n2 + 7 * n3)
    xd = _dev(x, prec)
    xr = xd.cpu().numpy().astype(np.complex128)            # the numbers the GPU transforms
    with pkg.FFT3(n1, n2, n3, prec) as f:
        X = f.forward(xd)
        back = f.inverse(X)
        Xh, bh = X.cpu().numpy().astype(np.complex128), back.cpu().numpy().astype(np.complex128)
    want = fo.fft3(xr)
    assert _rel(Xh, want) <= TOL[prec], _rel(Xh, want)
    want_back = fo.fft3(Xh, sign=1)
    assert _rel(bh, want_back) <= TOL[prec]
    assert _rel(bh, xr) <= 2 * TOL[prec]


@pytest.mark.parametrize("prec", ["c64", "c32"])
def test_in_place_equals_out_of_place_and_is_reproducible(pkg, prec):
    n1, n2, n3 = 128, 32, 64
    x = _dev(ji.fft_field(n1, n2, n3, seed=610), prec)
    with pkg.FFT3(n1, n2, n3, prec) as f:
        a = f.forward(x)
        b = x.clone()
        f.forward(b, out=b)
        c = f.forward(x)
        assert bool((a == b).all()) and bool((a == c).all())
        ia = f.inverse(a)
        f.inverse(b, out=b)
        assert bool((ia == b).all())


@pytest.mark.parametrize("prec", ["c64", "c32"])
@pytest.mark.parametrize("shape", [(64, 32, 16), (8, 256, 4), (256, 16, 32), (16, 16, 1024)])
def test_spectral_step_matches_oracle(pkg, shape, prec):
    import torch

    import oracle.fft as fo
    n1, n2, n3 = shape
    u0 = ji.fft_field(n1, n2, n3, seed=620 + n1)
    alpha, t = 1e-4, 3.0
    with pkg.FFT3(n1, n2, n3, prec) as f:
        U = f.forward(_dev(u0, prec))
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        u = f.evolve(U, alpha, t, energy=e)
        e2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        f.evolve(U, alpha, t, energy=e2)
        Uh = U.cpu().numpy().astype(np.complex128)
        uh = u.cpu().numpy().astype(np.complex128)
    want_u, want_e = fo.evolve(Uh, alpha, t)
    assert _rel(uh, want_u) <= TOL[prec], _rel(uh, want_u)
    assert abs(float(e.item()) - want_e) <= TOL[prec] * want_e
    assert float(e.item()) == float(e2.item())              # fixed-order reduction: bitwise repeatable
    # at t = 0 the step is the inverse transform
    with pkg.FFT3(n1, n2, n3, prec) as f:
        U = f.forward(_dev(u0, prec))
        assert bool((f.evolve(U, alpha, 0.0) == f.inverse(U)).all())


def test_bad_arguments(pkg):
    import torch
    with pytest.raises(pkg.JacError):
        pkg.FFT3(24, 16, 16, "c32")
    with pkg.FFT3(16, 8, 4, "c32") as f:
        x = torch.zeros((4, 8, 16), dtype=torch.complex64, device="cuda")
        with pytest.raises(ValueError):
            f.forward(torch.zeros((4, 8, 16), dtype=torch.complex128, device="cuda"))
        with pytest.raises(pkg.JacError):
            f.evolve(x, -1.0, 1.0)
        big = torch.zeros(2 * 4 * 8 * 16 + 8, dtype=torch.complex64, device="cuda")
        a, b = big[:512].view(4, 8, 16), big[8:520].view(4, 8, 16)      # overlapping, not equal
        with pytest.raises(pkg.JacError):
            f.forward(a, out=b)
