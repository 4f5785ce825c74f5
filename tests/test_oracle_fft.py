"""Pins for the oracle's own FFT (the first and last steps of Alg. 2).

Independent references: the O(m^2) DFT written out with exactly reduced phase
indices, numpy.fft (a library routine), and single-mode inputs whose transform
is known in closed form.
"""
import numpy as np
import pytest

LENGTHS = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 16, 18, 20, 24, 25, 27, 28, 32, 35, 40, 48, 49, 64, 70, 96,
           128, 140, 160, 192, 224, 256, 384, 512, 1024,
           # prime factors above 7 (padded lengths 2n of grids such as n = 11, 13, 17, 61, 101)
           11, 13, 22, 26, 34, 38, 46, 122, 202, 254]


def brute_dft(x, sign):
    m = len(x)
    j = np.arange(m)
    e = np.outer(j, j) % m  # exact phase index
    return (np.exp(sign * 2j * np.pi * e / m) * x[None, :]).sum(axis=1)


@pytest.mark.parametrize("m", LENGTHS)
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_vs_brute_force_and_numpy(oracle, m, sign):
    rng = np.random.default_rng(m)
    x = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    X = oracle.fft(x, sign)
    ref = np.fft.fft(x) if sign < 0 else m * np.fft.ifft(x)
    scale = np.abs(x).sum()
    assert np.abs(X - ref).max() <= 1e-14 * scale
    if m <= 256:
        assert np.abs(X - brute_dft(x, sign)).max() <= 1e-13 * scale


@pytest.mark.parametrize("m", [6, 64, 70, 192, 224, 1024])
def test_fft_single_mode_closed_form(oracle, m):
    # x_j = exp(+2 pi i j k0 / m)  =>  forward DFT = m at k0, 0 elsewhere
    for k0 in [0, 1, m // 3, m - 1]:
        j = np.arange(m)
        x = np.exp(2j * np.pi * ((j * k0) % m) / m)
        X = oracle.fft(x, -1)
        ref = np.zeros(m, complex)
        ref[k0] = m
        assert np.abs(X - ref).max() <= 1e-12 * m


def test_fft3_vs_numpy(oracle):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 8, 12)) + 1j * rng.standard_normal((6, 8, 12))
    assert np.abs(oracle.fft3(x, -1) - np.fft.fftn(x)).max() <= 1e-13 * np.abs(x).sum()
    assert np.abs(oracle.fft3(x, +1) - x.size * np.fft.ifftn(x)).max() <= 1e-13 * np.abs(x).sum()


def test_forward_spectrum_and_direct_coefficients(oracle):
    rng = np.random.default_rng(4)
    n = (5, 6, 4)
    rho = rng.standard_normal(n)
    S = oracle.forward_spectrum(rho)
    P = np.zeros((10, 12, 8))
    P[:5, :6, :4] = rho
    ref = np.fft.fftn(P)[:, :, :5]
    assert S.shape == ref.shape
    assert np.abs(S - ref).max() <= 1e-13 * np.abs(rho).sum()
    for k in [(0, 0, 0), (1, 2, 3), (9, 11, 4), (5, 6, 0)]:
        assert abs(oracle.dft_coeff(rho, k) - ref[k]) <= 1e-13 * np.abs(rho).sum()
