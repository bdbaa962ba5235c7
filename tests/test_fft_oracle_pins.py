"""Pins of the FP64 FFT oracle (oracle/fft_oracle.c) against facts the
mathematics fixes, not against the oracle itself:

  * a unit impulse at the origin transforms to all ones, exactly;
  * a single Fourier mode transforms to N at its frequency and 0 elsewhere;
  * Parseval: sum |x|^2 = sum |X|^2 / N;
  * the inverse undoes the forward transform;
  * linearity, and the shift theorem (a cyclic shift multiplies X by a phase);
  * real input gives a Hermitian spectrum, X[-k] = conj(X[k]);
  * the direct triple-sum 3-D DFT (one O(N) sum per output, not separated by
    axis), written out here, on tiny grids;
  * numpy.fft (a library routine the oracle does not use);
  * the spectral step on a single mode decays it by exactly
    exp(-4 pi^2 alpha t |kbar|^2), and at t = 0 it returns the field.

A plausible mistake in the oracle -- a wrong sign, a transposed axis stride,
a missing 1/N, an unsigned frequency in the step -- fails several of them.
"""
import numpy as np
import pytest

import jacobi_inputs as ji


@pytest.fixture(scope="module")
def fo():
    import oracle.fft as f
    f.build()
    return f


SHAPES = [(8, 4, 2), (16, 8, 4), (4, 16, 8), (32, 2, 16), (1, 8, 8), (6, 5, 3)]


def _mode(n1, n2, n3, a, b, c):
    z, y, x = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    return np.exp(2j * np.pi * (a * x / n1 + b * y / n2 + c * z / n3))


@pytest.mark.parametrize("shape", SHAPES)
def test_delta_transforms_to_ones(fo, shape):
    n1, n2, n3 = shape
    x = np.zeros((n3, n2, n1), complex)
    x[0, 0, 0] = 1.0
    X = fo.fft3(x)
    assert np.array_equal(X, np.ones_like(X))


@pytest.mark.parametrize("shape", SHAPES)
def test_single_mode_is_a_spike(fo, shape):
    n1, n2, n3 = shape
    a, b, c = n1 // 3, n2 - 1, n3 // 2
    X = fo.fft3(_mode(n1, n2, n3, a, b, c))
    want = np.zeros_like(X)
    want[c, b, a] = n1 * n2 * n3
    assert np.abs(X - want).max() <= 1e-12 * n1 * n2 * n3


@pytest.mark.parametrize("shape", SHAPES)
def test_parseval_and_round_trip(fo, shape):
    n1, n2, n3 = shape
    x = ji.fft_field(n1, n2, n3, seed=7)
    X = fo.fft3(x)
    N = n1 * n2 * n3
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(X) ** 2) / N) <= 1e-12 * np.sum(np.abs(x) ** 2)
    back = fo.fft3(X, sign=1)
    assert np.abs(back - x).max() <= 1e-13


def test_linearity_and_shift_theorem(fo):
    n1, n2, n3 = 16, 8, 4
    x = ji.fft_field(n1, n2, n3, seed=8)
    y = ji.fft_field(n1, n2, n3, seed=9)
    X, Y = fo.fft3(x), fo.fft3(y)
    Z = fo.fft3(2.5 * x - 1j * y)
    assert np.abs(Z - (2.5 * X - 1j * Y)).max() <= 1e-12 * np.abs(Z).max()
    s = (3, 5, 1)                                       # shift along x, y, z
    xs = np.roll(x, shift=(s[2], s[1], s[0]), axis=(0, 1, 2))
    kz, ky, kx = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    phase = np.exp(-2j * np.pi * (kx * s[0] / n1 + ky * s[1] / n2 + kz * s[2] / n3))
    assert np.abs(fo.fft3(xs) - phase * X).max() <= 1e-12 * np.abs(X).max()


def test_real_input_gives_hermitian_spectrum(fo):
    n1, n2, n3 = 8, 16, 4
    x = ji.fft_field(n1, n2, n3, seed=10).real.astype(complex)
    X = fo.fft3(x)
    neg = X[(-np.arange(n3)) % n3][:, (-np.arange(n2)) % n2][:, :, (-np.arange(n1)) % n1]
    assert np.abs(neg - np.conj(X)).max() <= 1e-12 * np.abs(X).max()


@pytest.mark.parametrize("shape", [(4, 2, 8), (3, 5, 2), (8, 8, 1)])
def test_direct_triple_sum(fo, shape):
    """The 3-D DFT as one sum over all N points per output (not separated by
    axis), written out with loops here."""
    n1, n2, n3 = shape
    x = ji.fft_field(n1, n2, n3, seed=11)
    want = np.zeros_like(x)
    for c in range(n3):
        for b in range(n2):
            for a in range(n1):
                acc = 0j
                for z in range(n3):
                    for y in range(n2):
                        for xx in range(n1):
                            acc += x[z, y, xx] * np.exp(-2j * np.pi * (a * xx / n1 + b * y / n2 + c * z / n3))
                want[c, b, a] = acc
    assert np.abs(fo.fft3(x) - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("shape", SHAPES)
def test_against_numpy_fft(fo, shape):
    n1, n2, n3 = shape
    x = ji.fft_field(n1, n2, n3, seed=12)
    X = fo.fft3(x)
    assert np.abs(X - np.fft.fftn(x)).max() <= 1e-12 * np.abs(X).max()
    assert np.abs(fo.fft3(X, sign=1) - np.fft.ifftn(X)).max() <= 1e-13
    # one axis alone, along each axis
    for axis, np_axis in ((0, 2), (1, 1), (2, 0)):
        assert np.abs(fo.dft_axis(x, axis) - np.fft.fft(x, axis=np_axis)).max() <= 1e-12 * np.abs(X).max()


@pytest.mark.parametrize("shape,mode", [((16, 8, 32), (3, 7, 30)), ((8, 8, 8), (4, 0, 5))])
def test_spectral_step_decays_a_single_mode_exactly(fo, shape, mode):
    n1, n2, n3 = shape
    a, b, c = mode
    u0 = _mode(n1, n2, n3, a, b, c)
    U = fo.fft3(u0)
    alpha, t = 1e-3, 2.0
    kb = [k if k < (n + 1) // 2 else k - n for k, n in ((a, n1), (b, n2), (c, n3))]
    decay = np.exp(-4 * np.pi ** 2 * alpha * t * sum(k * k for k in kb))
    u, energy = fo.evolve(U, alpha, t)
    assert np.abs(u - decay * u0).max() <= 1e-12
    N = n1 * n2 * n3
    assert abs(energy - N * decay ** 2) <= 1e-12 * N * decay ** 2
    u_0, e_0 = fo.evolve(U, alpha, 0.0)
    assert np.abs(u_0 - u0).max() <= 1e-13 and abs(e_0 - N) <= 1e-11 * N


def test_spectral_step_uses_signed_frequencies(fo):
    """Modes k and n - k are the same physical wave number: they decay alike."""
    n1, n2, n3 = 16, 4, 4
    alpha, t = 2e-3, 1.0
    rates = []
    for a in (3, 13):
        U = fo.fft3(_mode(n1, n2, n3, a, 0, 0))
        _, e = fo.evolve(U, alpha, t)
        rates.append(e)
    assert abs(rates[0] - rates[1]) <= 1e-12 * rates[0]
    assert rates[0] < n1 * n2 * n3                       # it did decay


@pytest.mark.parametrize("shape", [(8, 4, 2), (16, 8, 4), (6, 5, 3)])
def test_single_point_form_equals_the_transform(fo, shape):
    """The one-output form used for sampled checks of large grids gives the
    transform's value at every index (forward and unscaled inverse)."""
    n1, n2, n3 = shape
    x = ji.fft_field(n1, n2, n3, seed=13)
    X = fo.fft3(x)
    Xi = fo.fft3(x, sign=1) * (n1 * n2 * n3)
    for kz in range(n3):
        for ky in range(n2):
            for kx in range(n1):
                assert abs(fo.point(x, (kx, ky, kz)) - X[kz, ky, kx]) <= 1e-12 * np.abs(X).max()
    assert abs(fo.point(x, (1, 2, 0), sign=1) - Xi[0, 2, 1]) <= 1e-12 * np.abs(Xi).max()
