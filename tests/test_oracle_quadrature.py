"""Pins for the GS table (eq. sin_1_x, Fig. 1) and the 1D integrals of eq. (Gten_sep).

References: the exact target 1/(8 pi r) evaluated against the table in
arbitrary precision (mpmath); closed forms of the 1D integrals at kappa = 0,
as alpha -> 0, and in the full-line limit of large alpha; mpmath quadrature
in the mid range.
"""
import math

import mpmath as mp
import numpy as np
import pytest


def test_gs_table_relative_accuracy_mpmath(oracle):
    # Fig. 1: double-precision accuracy of the GS approximation on (1e-4, delta].
    eps, delta = 1e-4, 2.0 * math.sqrt(3.0)
    w, a = oracle.gs_table(eps, delta)
    assert 400 <= len(w) <= 700  # the paper uses S = 460; this construction gives about 530
    mp.mp.dps = 40
    W = [mp.mpf(float(x)) for x in w]
    A = [mp.mpf(float(x)) for x in a]
    worst = 0.0
    for r in np.geomspace(eps * 1.0001, delta, 60):
        rr = mp.mpf(float(r))
        s = mp.fsum(Wi * mp.exp(-Ai * rr * rr) for Wi, Ai in zip(W, A))
        worst = max(worst, float(abs(8 * mp.pi * rr * s - 1)))
    assert worst <= 2e-15, worst


def test_gs_ratio_long_double_matches_mpmath(oracle):
    w, a = oracle.gs_table(1e-4, 3.0)
    for r in [1.2e-4, 1e-2, 0.5, 2.9]:
        assert abs(oracle.gs_ratio(r, w, a) - 1.0) <= 2e-15


def test_gs_table_closed_form_entries(oracle):
    # tau_s on a uniform grid of step h_tau: a_{s+1}/a_s = exp(2 h), w_{s+1}/w_s = exp(h),
    # and w_s^2 / a_s = ((1/(8 pi)) (2/sqrt(pi)) h)^2 for every s.
    h = 0.1
    w, a = oracle.gs_table(1e-4, 5.0, h)
    np.testing.assert_allclose(a[1:] / a[:-1], math.exp(2 * h), rtol=1e-13)
    np.testing.assert_allclose(w[1:] / w[:-1], math.exp(h), rtol=1e-13)
    c = (1 / (8 * math.pi)) * (2 / math.sqrt(math.pi)) * h
    np.testing.assert_allclose(w * w / a, c * c, rtol=1e-13)


@pytest.mark.parametrize("alpha", [1e-30, 1e-3, 0.1, 1.0, 10.0, 100.0, 1e4, 1e6, 1e9])
def test_integrals_kappa_zero_closed_form(oracle, alpha):
    L = 4.0634920634920634
    G, H = oracle.integrals_1d(alpha, L, 0.0)
    # closed forms, evaluated in 50-digit arithmetic (the H form cancels for small alpha)
    mp.mp.dps = 50
    al, LL = mp.mpf(alpha), mp.mpf(L)
    sa = mp.sqrt(al)
    Ge = mp.sqrt(mp.pi / al) * mp.erf(sa * LL)
    He = mp.sqrt(mp.pi) / (2 * al * sa) * mp.erf(sa * LL) - LL * mp.exp(-al * LL * LL) / al
    assert abs(G - float(Ge)) <= 2e-15 * abs(float(Ge))
    assert abs(H - float(He)) <= 2e-15 * abs(float(He))


@pytest.mark.parametrize("k", [1, 2, 7, 31, 64, 257])
def test_integrals_vanishing_alpha_closed_form(oracle, k):
    # alpha -> 0: G = 2 sin(kL)/k, H = 2 [L^2 sin(kL)/k + 2 L cos(kL)/k^2 - 2 sin(kL)/k^3]
    L = 2.5
    kap = math.pi * k / L
    G, H = oracle.integrals_1d(1e-40, L, kap)
    s, c = math.sin(kap * L), math.cos(kap * L)
    Ge = 2 * s / kap
    He = 2 * (L * L * s / kap + 2 * L * c / kap ** 2 - 2 * s / kap ** 3)
    assert abs(G - Ge) <= 2e-15 * 2 * L
    assert abs(H - He) <= 2e-15 * 2 * L ** 3 / 3


@pytest.mark.parametrize("alpha", [1e3, 1e5, 1e8, 1e10])
@pytest.mark.parametrize("k", [0, 1, 13, 128, 512])
def test_integrals_large_alpha_full_line(oracle, alpha, k):
    # alpha L^2 >> 1: the window cut is below 1e-300; full-line Gaussian transforms hold.
    L = 2.0 * 128 / 127
    kap = math.pi * k / L
    G, H = oracle.integrals_1d(alpha, L, kap)
    ex = math.exp(-kap * kap / (4 * alpha))
    Ge = math.sqrt(math.pi / alpha) * ex
    He = math.sqrt(math.pi) / (2 * alpha ** 1.5) * (1 - kap * kap / (2 * alpha)) * ex
    assert abs(G - Ge) <= 2e-15 * math.sqrt(math.pi / alpha)
    assert abs(H - He) <= 2e-15 * math.sqrt(math.pi) / (2 * alpha ** 1.5)


@pytest.mark.parametrize("alpha,k", [(0.05, 3), (0.7, 20), (2.0, 1), (6.0, 45), (9.0, 100)])
def test_integrals_mid_range_mpmath(oracle, alpha, k):
    L = 2.5
    kap = math.pi * k / L
    G, H = oracle.integrals_1d(alpha, L, kap)
    mp.mp.dps = 30
    f0 = lambda y: mp.exp(-alpha * y * y) * mp.cos(kap * y)
    pts = [mp.mpf(L) * i / (2 * k + 2) for i in range(2 * k + 3)]
    Ge = 2 * mp.quad(f0, pts)
    He = 2 * mp.quad(lambda y: y * y * f0(y), pts)
    m0 = math.sqrt(math.pi / alpha) / 2 * math.erf(math.sqrt(alpha) * L)
    assert abs(G - float(Ge)) <= 2e-15 * 2 * m0
    assert abs(H - float(He)) <= 2e-15 * 2 * L * L * m0
