"""Pins of the oracle's DFT: direct sum, a library FFT it does not call,
Parseval and inversion."""
import cmath

import numpy as np
import pytest

from oracle import dft


def _direct_dft2(x):
    N = x.shape[0]
    out = np.zeros((N, N), dtype=np.complex128)
    for q0 in range(N):
        for q1 in range(N):
            s = 0j
            for r0 in range(N):
                for r1 in range(N):
                    s += x[r0, r1] * cmath.exp(-2j * cmath.pi * (q0 * r0 + q1 * r1) / N)
            out[q0, q1] = s
    return out


def _rand(rng, N):
    return rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))


def test_direct_sum_8x8():
    rng = np.random.default_rng(1)
    x = _rand(rng, 8)
    np.testing.assert_allclose(dft.fft2(x), _direct_dft2(x), rtol=0, atol=1e-12)


def test_direct_sum_non_symmetric_impulse():
    # an off-centre impulse fixes the sign and the axis order of the exponent
    x = np.zeros((8, 8), dtype=np.complex128)
    x[1, 3] = 1.0
    q = np.arange(8)
    expect = np.exp(-2j * np.pi * (q[:, None] * 1 + q[None, :] * 3) / 8)
    np.testing.assert_allclose(dft.fft2(x), expect, atol=1e-14)


@pytest.mark.parametrize("N", [8, 64, 128])
def test_matches_library_fft(N):
    rng = np.random.default_rng(N)
    x = _rand(rng, N)
    X = dft.fft2(x)
    ref = np.fft.fft2(x)
    assert np.abs(X - ref).max() <= 1e-11 * np.abs(ref).max()
    np.testing.assert_allclose(dft.ifft2(ref), np.fft.ifft2(ref), atol=1e-12 * np.abs(x).max())


@pytest.mark.parametrize("N", [8, 64])
def test_parseval_and_inverse(N):
    rng = np.random.default_rng(7 + N)
    x = _rand(rng, N)
    X = dft.fft2(x)
    np.testing.assert_allclose((np.abs(X) ** 2).sum(), N * N * (np.abs(x) ** 2).sum(), rtol=1e-12)
    np.testing.assert_allclose(dft.ifft2(X), x, atol=1e-12)
