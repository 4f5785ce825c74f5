"""Pins for the oracle solve (Alg. 2): brute-force convolution, the paper's
printed errors (Tab. 1, 4-9, fixtures in tests/golden/), and exact solutions of
the benchmark densities."""
import math

import numpy as np
import pytest

from paper_2506_04489_gb300 import workloads as W
from tests import analytic as A


def brute_solve(M, rho):
    """u_x = sum_{x'} K(x - x' mod 2n) rho_x' with K(j) = (1/N) sum_k M(|k|) exp(2 pi i k.j/2n)."""
    n = rho.shape
    m = [2 * p for p in n]
    K = np.zeros(m)
    kk = [np.minimum(np.arange(mp), mp - np.arange(mp)) for mp in m]
    for j0 in range(m[0]):
        for j1 in range(m[1]):
            for j2 in range(m[2]):
                acc = 0.0
                for a0 in range(m[0]):
                    for a1 in range(m[1]):
                        ph = (a0 * j0) / m[0] + (a1 * j1) / m[1]
                        for a2 in range(m[2]):
                            acc += M[kk[0][a0], kk[1][a1], kk[2][a2]] * math.cos(
                                2 * math.pi * (ph + (a2 * j2) / m[2]))
                K[j0, j1, j2] = acc / (m[0] * m[1] * m[2])
    u = np.zeros(n)
    for x in np.ndindex(*n):
        s = 0.0
        for y in np.ndindex(*n):
            s += K[(x[0] - y[0]) % m[0], (x[1] - y[1]) % m[1], (x[2] - y[2]) % m[2]] * rho[y]
        u[x] = s
    return u


@pytest.mark.parametrize("n", [(3, 3, 3), (3, 4, 5), (2, 5, 3)])
def test_solve_matches_brute_force_convolution(oracle, n):
    rng = np.random.default_rng(sum(n))
    M = rng.uniform(0.5, 2.0, size=tuple(p + 1 for p in n))
    rho = rng.standard_normal(n)
    u = oracle.solve(M, rho)
    ref = brute_solve(M, rho)
    assert np.abs(u - ref).max() <= 1e-13 * np.abs(ref).max()


def _check_row(E, E_paper, floor=False):
    """Resolution-limited rows must match the paper to 2%; at the rounding floor
    (E below 1e-11, or no 10x gain at the next grid in the paper's own table)
    only the order of magnitude is reproducible."""
    if E_paper >= 1e-11 and not floor:
        assert abs(E / E_paper - 1.0) <= 0.02, (E, E_paper)
    else:
        assert E <= 10.0 * max(E_paper, 1e-14), (E, E_paper)


def _rows(name, nmax):
    """Rows with n <= nmax, each with a flag telling whether it is a floor row."""
    rows = A.read_table(name)
    out = []
    for i, r in enumerate(rows):
        if r[-2] > nmax:
            continue
        nxt = rows[i + 1] if i + 1 < len(rows) and rows[i + 1][:-2] == r[:-2] else None
        floor = nxt is not None and nxt[-1] > 0.1 * r[-1]
        out.append(r + (floor,))
    return out


@pytest.mark.parametrize("sigma,n,E_paper,floor", _rows("tab1_gaussian.txt", 64))
def test_table1_gaussian(oracle, sigma, n, E_paper, floor):
    n = int(n)
    lo, hi = -2.0, 2.0
    _, _, M = oracle.plan_tables(n, lo, hi)
    u = oracle.solve(M, W.gaussian(n, lo, hi, sigma))
    _check_row(A.rel_err(u, A.gaussian_u(n, lo, hi, sigma)), E_paper, floor)


@pytest.mark.parametrize("n,E_paper,floor", _rows("tab4_gaussian_rect.txt", 64))
def test_table4_gaussian_rectangular(oracle, n, E_paper, floor):
    n = int(n)
    lo, hi = (-3.0, -2.0, -1.0), (2.0, 3.5, 5.0)
    c = tuple((a + b) / 2 for a, b in zip(lo, hi))
    _, _, M = oracle.plan_tables(n, lo, hi)
    u = oracle.solve(M, W.gaussian(n, lo, hi, 0.2, c))
    _check_row(A.rel_err(u, A.gaussian_u(n, lo, hi, 0.2, c)), E_paper, floor)


@pytest.mark.parametrize("n,E_paper,floor", _rows("tab5_two_gaussians.txt", 64))
def test_table5_two_gaussians(oracle, n, E_paper, floor):
    n = int(n)
    lo, hi = -2.0, 2.0
    c, d = (0.0, 0.0, 0.0), (0.1, -0.05, 0.05)
    _, _, M = oracle.plan_tables(n, lo, hi)
    u = oracle.solve(M, W.two_gaussians(n, lo, hi, 0.2, 0.1, c, d))
    _check_row(A.rel_err(u, A.two_gaussians_u(n, lo, hi, 0.2, 0.1, c, d)), E_paper, floor)


@pytest.mark.parametrize("n,E_paper,floor", _rows("tab6_bump_rect.txt", 64))
def test_table6_bump_rectangular(oracle, n, E_paper, floor):
    n = int(n)
    lo, hi = (-3.0, -2.0, -2.0), (1.0, 3.0, 4.0)
    c = tuple((a + b) / 2 for a, b in zip(lo, hi))
    _, _, M = oracle.plan_tables(n, lo, hi)
    u = oracle.solve(M, W.paper_bump(n, lo, hi, 2.0, 10.0, c))
    _check_row(A.rel_err(u, A.bump_u(n, lo, hi, 2.0, 10.0, c)), E_paper, floor)


@pytest.mark.parametrize("n,E_paper,floor", _rows("tab7_anisotropic.txt", 64))
def test_table7_anisotropic(oracle, n, E_paper, floor):
    n = int(n)
    lo, hi = -2.0, 2.0
    sig = (0.30, 0.20, 0.28)
    _, _, M = oracle.plan_tables(n, lo, hi)
    u = oracle.solve(M, W.anisotropic(n, lo, hi, sig))
    _check_row(A.rel_err(u, A.anisotropic_u(n, lo, hi, sig)), E_paper, floor)


@pytest.mark.parametrize("Lf,n,E_paper,floor", [r for r in _rows("tab8_flat.txt", 64) if r[0] in (2, 8, 32)])
def test_table8_flat_domains(oracle, Lf, n, E_paper, floor):
    n = int(n)
    lo, hi = (-2.0, -2 * Lf, -2 * Lf), (2.0, 2 * Lf, 2 * Lf)
    sig = (0.2, 0.2 * Lf, 0.2 * Lf)
    _, _, M = oracle.plan_tables(n, lo, hi)
    u = oracle.solve(M, W.anisotropic(n, lo, hi, sig))
    _check_row(A.rel_err(u, A.anisotropic_u(n, lo, hi, sig)), E_paper, floor)


@pytest.mark.parametrize("n,E_paper,floor", _rows("tab9_oscillating.txt", 64))
def test_table9_oscillating(oracle, n, E_paper, floor):
    n = int(n)
    lo, hi = -2.0, 2.0
    _, _, M = oracle.plan_tables(n, lo, hi)
    u = oracle.solve(M, W.oscillating(n, lo, hi, 0.3, 20.0))
    _check_row(A.rel_err(u, A.oscillating_u(n, lo, hi, 0.3, 20.0)), E_paper, floor)


@pytest.mark.slow
def test_table1_gaussian_128(oracle):
    lo, hi, sigma = -2.0, 2.0, 0.2
    _, _, M = oracle.plan_tables(128, lo, hi)
    u = oracle.solve(M, W.gaussian(128, lo, hi, sigma))
    _check_row(A.rel_err(u, A.gaussian_u(128, lo, hi, sigma)), 3.859e-15)


def test_unit_box_gaussian_scale_invariance(oracle):
    # [-1,1]^3 with sigma = 0.1 is Tab. 1's [-2,2]^3, sigma = 0.2 row scaled by 1/2:
    # the relative error must match that row (4.154e-9 at n = 32).
    lo, hi = -1.0, 1.0
    _, _, M = oracle.plan_tables(32, lo, hi)
    u = oracle.solve(M, W.gaussian(32, lo, hi, 0.1))
    _check_row(A.rel_err(u, A.gaussian_u(32, lo, hi, 0.1)), 4.154e-9)


def test_prescribed_bump_unit_box(oracle):
    # eq. (bump) with d = 1, R = 0.8 on [-1,1]^3: u* is exactly the C-infinity bump
    # profile used as a density in the large-grid workloads; convergence in n.
    lo, hi = -1.0, 1.0
    errs = []
    for n in (32, 64):
        _, _, M = oracle.plan_tables(n, lo, hi)
        u = oracle.solve(M, W.paper_bump(n, lo, hi, 0.8, 1.0))
        errs.append(A.rel_err(u, A.bump_u(n, lo, hi, 0.8, 1.0)))
    # the density (-Laplacian of a bump) has Fourier coefficients decaying like
    # exp(-c sqrt(k)): 1.1e-2 at n = 32 and 4.6e-4 at n = 64
    assert errs[1] < errs[0] / 10
    assert errs[1] < 1e-3


def test_bump_profile_density_radial_quadrature(oracle):
    # The C-infinity bump exp(-1/(1 - r^2/0.64)) as a density: exact potential by 1D
    # radial quadrature (Newton's shell theorem) on the grid's distinct radii.
    lo, hi, n, R = -1.0, 1.0, 64, 0.8
    _, _, M = oracle.plan_tables(n, lo, hi)
    rho = W.bump_profile(n, lo, hi, R)
    u = oracle.solve(M, rho)
    X, Y, Z = W.mesh(n, lo, hi)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    prof = lambda s: math.exp(-1.0 / (1.0 - s * s / (R * R))) if s < R else 0.0
    rs = np.round(r, 12)
    uniq = np.unique(rs)
    sample = uniq[:: max(1, len(uniq) // 150)]
    ref = {float(q): A.radial_potential(prof, R, float(q)) for q in sample}
    umax = max(abs(v) for v in ref.values())
    worst = 0.0
    for q, v in ref.items():
        worst = max(worst, float(np.abs(u[rs == q] - v).max()))
    # the bump is C-infinity but not analytic: 1.2e-7 at n = 64 on [-1,1]^3
    assert worst / umax < 5e-7, worst / umax


def _order(eps, E):
    return math.log(E[0] / E[-1]) / math.log(eps[0] / eps[-1])


def test_cutoff_error_orders_superpotential_vs_plain_gs(oracle):
    # Lemma 1 / Thm. 1: the super-potential kernel's GS cutoff error is O(eps^4); the
    # original GS method without near-field correction (Tab. 2 brackets) is O(eps^2).
    # Absolute values depend on the unstated GS generator and eps convention of the
    # paper's code (Tab. 3 is not reproduced); the orders are.
    lo, hi, sigma = -2.0, 2.0, 0.2
    eps = [2.2e-2, 5.7e-3, 1.6e-3]
    E4 = []
    for e in eps:
        _, _, M = oracle.plan_tables(64, lo, hi, eps=e)
        E4.append(A.rel_err(oracle.solve(M, W.gaussian(64, lo, hi, sigma)), A.gaussian_u(64, lo, hi, sigma)))
    assert 3.5 <= _order(eps, E4) <= 4.5, E4
    eps2 = [7.5e-2, 5.7e-3, 4.7e-4]
    E2 = []
    for e in eps2:
        _, _, M = oracle.plan_tables(32, lo, hi, eps=e, kernel="gs_plain")
        E2.append(A.rel_err(oracle.solve(M, W.gaussian(32, lo, hi, sigma)), A.gaussian_u(32, lo, hi, sigma)))
    assert 1.7 <= _order(eps2, E2) <= 2.3, E2


def test_spectral_laplacian_invariant(oracle):
    # The density is formed from a compactly supported C-infinity u* (the bump
    # exp(-1/(1 - r^2/0.64)) on [-1,1]^3) by the Laplacian taken spectrally on the
    # padded periodic grid (rho_hat = |kappa|^2 u_hat, kappa = pi k / L): the solve must
    # return u* up to the method's own discretisation error, converging with n.  A wrong
    # wavenumber scale, a sign, or a dropped term of the multiplier gives O(1) errors.
    lo, hi = -1.0, 1.0
    errs = []
    for n in (32, 64):
        _, L = oracle.geometry((n,) * 3, (lo,) * 3, (hi,) * 3)
        ustar = W.bump_profile(n, lo, hi, 0.8)
        m = 2 * n
        P = np.zeros((m, m, m))
        P[:n, :n, :n] = ustar
        k = np.fft.fftfreq(m, 1.0 / m)  # signed wavenumbers of the padded axis
        kap = [math.pi * k / L[p] for p in range(3)]
        K2 = kap[0][:, None, None] ** 2 + kap[1][None, :, None] ** 2 + kap[2][None, None, :] ** 2
        rho = np.real(np.fft.ifftn(K2 * np.fft.fftn(P)))[:n, :n, :n]
        _, _, M = oracle.plan_tables(n, lo, hi)
        errs.append(A.rel_err(oracle.solve(M, rho), ustar))
    # measured: 2.9e-4 at n = 32, 1.5e-5 at n = 64 (about h^4)
    assert errs[0] < 1e-3
    assert errs[1] < 5e-5 and errs[1] < errs[0] / 8
