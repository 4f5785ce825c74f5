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
    G, H = oracle.integrals_1d(alpha, L, 0)
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
    # alpha -> 0: G = 2 sin(kL)/k = 0 (kL = pi k), H = 4 L (-1)^k / kappa^2
    L = 2.5
    kap = math.pi * k / L
    G, H = oracle.integrals_1d(1e-40, L, k)
    He = 4 * L * (-1) ** k / kap ** 2
    assert abs(G) <= 1e-30
    assert abs(H - He) <= 2e-15 * abs(He)


@pytest.mark.parametrize("alpha", [1e3, 1e5, 1e8, 1e10])
@pytest.mark.parametrize("k", [0, 1, 13, 128, 512])
def test_integrals_large_alpha_full_line(oracle, alpha, k):
    # alpha L^2 >> 1: the window cut is below 1e-300; full-line Gaussian transforms hold.
    L = 2.0 * 128 / 127
    kap = math.pi * k / L
    G, H = oracle.integrals_1d(alpha, L, k)
    ex = math.exp(-kap * kap / (4 * alpha))
    Ge = math.sqrt(math.pi / alpha) * ex
    He = math.sqrt(math.pi) / (2 * alpha ** 1.5) * (1 - kap * kap / (2 * alpha)) * ex
    assert abs(G - Ge) <= 2e-15 * math.sqrt(math.pi / alpha)
    assert abs(H - He) <= 2e-15 * math.sqrt(math.pi) / (2 * alpha ** 1.5)


def _mp_reference(alpha, L, k):
    mp.mp.dps = 40
    al, LL = mp.mpf(alpha), mp.mpf(L)
    kap = mp.pi * k / LL
    f0 = lambda y: mp.exp(-al * y * y) * mp.cos(kap * y)
    pts = [LL * i / (2 * k + 2) for i in range(2 * k + 3)]
    return 2 * mp.quad(f0, pts), 2 * mp.quad(lambda y: y * y * f0(y), pts)


def _fourth_scale(alpha, L, k):
    """int_0^L |P4| dy / kappa^4 for P = f and P = g (P4: fourth derivative): the size
    of the remainder left after two integrations by parts, the accuracy scale of that form."""
    mp.mp.dps = 30
    al, LL = mp.mpf(alpha), mp.mpf(L)
    kap4 = (mp.pi * k / LL) ** 4
    f4 = lambda y: abs((16 * al ** 4 * y ** 4 - 48 * al ** 3 * y ** 2 + 12 * al ** 2) * mp.exp(-al * y * y))
    g4 = lambda y: abs((16 * al ** 4 * y ** 6 - 112 * al ** 3 * y ** 4 + 156 * al ** 2 * y ** 2 - 24 * al)
                       * mp.exp(-al * y * y))
    pts = mp.linspace(0, LL, 40)
    return float(mp.quad(f4, pts) / kap4), float(mp.quad(g4, pts) / kap4)


@pytest.mark.parametrize("alpha,k", [(0.05, 3), (0.7, 20), (2.0, 1), (6.0, 45), (9.0, 100), (40.0, 2)])
def test_integrals_mid_range_mpmath(oracle, alpha, k):
    L = 2.5
    G, H = oracle.integrals_1d(alpha, L, k)
    Ge, He = _mp_reference(alpha, L, k)
    kap = math.pi * k / L
    if kap * kap < 4 * alpha:  # direct form: accurate to the integrand's size
        m0 = math.sqrt(math.pi / alpha) / 2 * math.erf(math.sqrt(alpha) * L)
        assert abs(G - float(Ge)) <= 2e-15 * 2 * m0
        assert abs(H - float(He)) <= 2e-15 * 2 * L * L * m0
    else:  # by-parts form: accurate to the result plus the remainder's size
        s0, s2 = _fourth_scale(alpha, L, k)
        assert abs(G - float(Ge)) <= 1e-14 * (abs(float(Ge)) + 2 * s0)
        assert abs(H - float(He)) <= 1e-14 * (abs(float(He)) + 2 * s2)


@pytest.mark.parametrize("alpha", [1e-3, 0.08, 0.5])
@pytest.mark.parametrize("k", [9, 26, 64, 200])
def test_integrals_relative_accuracy_high_k(oracle, alpha, k):
    # Wide Gaussians (a L^2 < 4) at high wavenumber: G and H fall far below the size of
    # their integrands, and the by-parts form still gives them to a few ulp.
    L = 2.0645161290322580
    G, H = oracle.integrals_1d(alpha, L, k)
    Ge, He = _mp_reference(alpha, L, k)
    assert abs(G - float(Ge)) <= 1e-14 * abs(float(Ge)), (G, float(Ge))
    assert abs(H - float(He)) <= 1e-14 * abs(float(He)), (H, float(He))


def test_multiplier_high_k_relative_accuracy_mpmath(oracle):
    # eqs. Gten_sep / convtheorem with a short GS table whose exponents span the direct,
    # by-parts and large-exponent regimes: M at high wavenumbers, where the GS sum
    # cancels, against every integral in 30-digit arithmetic.
    L, n = 2.0, 16
    a = np.geomspace(1e-3, 2e3, 14)
    w = np.geomspace(1e-3, 1.0, 14)
    M = oracle.multiplier((n, n, n), (L, L, L), w, a)
    mp.mp.dps = 30
    LL = mp.mpf(L)
    cache = {}

    def gh(s, k):
        if (s, k) not in cache:
            al = mp.mpf(a[s])
            kap = mp.pi * k / LL
            f0 = lambda y: mp.exp(-al * y * y) * mp.cos(kap * y)
            pts = sorted(set([LL * i / (2 * k + 2) for i in range(2 * k + 3)]
                             + [min(LL, mp.mpf(c) / mp.sqrt(al)) for c in (0.5, 1, 2, 4)]))
            cache[(s, k)] = (2 * mp.quad(f0, pts), 2 * mp.quad(lambda y: y * y * f0(y), pts))
        return cache[(s, k)]

    for k in [(16, 0, 0), (11, 7, 16), (16, 16, 16), (3, 14, 9)]:
        V = mp.mpf(0)
        for s in range(len(a)):
            g = [gh(s, kk) for kk in k]
            V += mp.mpf(w[s]) * (g[0][1] * g[1][0] * g[2][0] + g[0][0] * g[1][1] * g[2][0]
                                 + g[0][0] * g[1][0] * g[2][1])
        ref = float(-sum((mp.pi * kk / LL) ** 2 for kk in k) * V)
        assert abs(M[k] - ref) <= 1e-13 * abs(ref), (k, M[k], ref)
