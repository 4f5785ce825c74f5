"""Pins for the multiplier M_k = -|kappa|^2 Vhat_k (eqs. convtheorem, Gten_sep).

The separable assembly is checked against the un-separated 3D Fourier integral
of V_GS(y) = sum_s w_s |y|^2 exp(-a_s |y|^2) over the window (eq. gs_x),
computed by a tensor Gauss-Legendre rule in numpy, on an anisotropic tiny
case so that a swapped axis, a dropped rank-3 term or a wrong wavenumber
scaling fails.
"""
import math

import numpy as np
import pytest


def brute_vhat(k, L, w, a, q=72):
    xg, wg = np.polynomial.legendre.leggauss(q)
    ys = [Lp * xg for Lp in L]
    ws = [Lp * wg for Lp in L]
    Y0, Y1, Y2 = np.meshgrid(*ys, indexing="ij")
    W3 = ws[0][:, None, None] * ws[1][None, :, None] * ws[2][None, None, :]
    r2 = Y0 ** 2 + Y1 ** 2 + Y2 ** 2
    kap = [math.pi * kp / Lp for kp, Lp in zip(k, L)]
    ph = np.cos(kap[0] * Y0 + kap[1] * Y1 + kap[2] * Y2)
    V = sum(ws_ * r2 * np.exp(-as_ * r2) for ws_, as_ in zip(w, a))
    return float((W3 * V * ph).sum()), kap


def test_multiplier_matches_3d_fourier_integral(oracle):
    n = (3, 4, 2)
    L = (1.0, 1.3, 0.8)
    w = np.array([0.3, 0.5, 0.2, 0.05])
    a = np.array([0.4, 2.0, 7.0, 30.0])
    M = oracle.multiplier(n, L, w, a)
    assert M.shape == (4, 5, 3)
    scale = np.abs(M).max()
    for k0 in range(4):
        for k1 in range(5):
            for k2 in range(3):
                V, kap = brute_vhat((k0, k1, k2), L, w, a)
                ref = -(kap[0] ** 2 + kap[1] ** 2 + kap[2] ** 2) * V
                assert abs(M[k0, k1, k2] - ref) <= 1e-12 * scale, (k0, k1, k2, M[k0, k1, k2], ref)


def test_multiplier_zero_mode_and_symmetry(oracle):
    w, a = oracle.gs_table(1e-4, 6.0)
    M = oracle.multiplier((8, 8, 8), (2.0, 2.0, 2.0), w, a)
    assert M[0, 0, 0] == 0.0
    # a cube: M is symmetric under any permutation of the three wavenumbers
    np.testing.assert_allclose(M, M.transpose(1, 0, 2), rtol=1e-13, atol=1e-16 * np.abs(M).max())
    np.testing.assert_allclose(M, M.transpose(2, 1, 0), rtol=1e-13, atol=1e-16 * np.abs(M).max())


@pytest.mark.parametrize("n,lo,hi", [((32, 32, 32), (-1, -1, -1), (1, 1, 1)),
                                     ((24, 32, 20), (-1, -2, -0.5), (1.5, 1, 1))])
def test_multiplier_asymptote(oracle, n, lo, hi):
    # Away from the axes (every |k_p| >= 4) the window and the GS cutoff barely matter
    # and M tends to the Fourier transform of the Newton kernel 1/(4 pi |x|): M |kappa|^2
    # -> 1 (a loose asymptote, but one no plausible mistake satisfies).  A wrong kappa scale, a missing normalisation or a
    # dropped rank-3 term of V_hat moves the ratio far from 1.
    _, L = oracle.geometry(n, lo, hi)
    _, _, M = oracle.plan_tables(n, lo, hi)
    k = [np.arange(m + 1) for m in n]
    kap2 = ((math.pi * k[0] / L[0]) ** 2)[:, None, None] + ((math.pi * k[1] / L[1]) ** 2)[None, :, None] + \
        ((math.pi * k[2] / L[2]) ** 2)[None, None, :]
    kmin = np.minimum(np.minimum(k[0][:, None, None], k[1][None, :, None]), k[2][None, None, :])
    r = (M * kap2)[kmin >= 4]
    assert np.median(np.abs(r - 1)) < 2e-3
    assert np.abs(r - 1).max() < 0.05
