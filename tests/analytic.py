"""Exact solutions printed in the paper, used as pins for the oracle and the GPU path.

Each function returns u* on the grid x_j = lo + j (hi - lo)/(n - 1).
"""
import math

import numpy as np
from scipy import integrate
from scipy.special import erf

from paper_2506_04489_gb300 import workloads as W


def gaussian_u(n, lo, hi, sigma, c=(0.0, 0.0, 0.0)):
    """u* = erf(r/(sqrt(2) sigma)) / (4 pi r), r = |x - c|  (Sec. 3.1, after eq. gaussian);
    its r -> 0 limit is 1/((2 pi)^{3/2} sigma)."""
    X, Y, Z = W.mesh(n, lo, hi)
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    safe = np.where(r > 0, r, 1.0)
    return np.where(r > 0, erf(r / (math.sqrt(2.0) * sigma)) / (4 * math.pi * safe),
                    1.0 / ((2 * math.pi) ** 1.5 * sigma))


def two_gaussians_u(n, lo, hi, sigma1, sigma2, c, d):
    c, d = np.asarray(c, float), np.asarray(d, float)
    return 0.5 * (gaussian_u(n, lo, hi, sigma1, c + d) + gaussian_u(n, lo, hi, sigma2, c - d))


def bump_u(n, lo, hi, R, d, c=(0.0, 0.0, 0.0)):
    """u* = exp(-d/(1 - |x-c|^2/R^2)) inside the ball, 0 outside (Sec. 3.2)."""
    X, Y, Z = W.mesh(n, lo, hi)
    r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
    out = np.zeros_like(r2)
    m = r2 < R * R
    out[m] = np.exp(-d / (1.0 - r2[m] / (R * R)))
    return out


def anisotropic_u(n, lo, hi, sig, c=(0.0, 0.0, 0.0)):
    X, Y, Z = W.mesh(n, lo, hi)
    return np.exp(-(X - c[0]) ** 2 / sig[0] ** 2 - (Y - c[1]) ** 2 / sig[1] ** 2
                  - (Z - c[2]) ** 2 / sig[2] ** 2)


def oscillating_u(n, lo, hi, sigma, omega, c=(0.0, 0.0, 0.0)):
    X, Y, Z = W.mesh(n, lo, hi)
    r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
    return np.exp(-r2 / sigma ** 2) * np.cos(omega * r2)


def radial_potential(rho_of_r, R, r):
    """Potential of a radial density supported in r < R by 1D quadrature:
    u(r) = (1/r) int_0^r rho(s) s^2 ds + int_r^R rho(s) s ds  (Newton's shell theorem)."""
    r = float(r)
    inner = integrate.quad(lambda s: rho_of_r(s) * s * s, 0.0, min(r, R), epsabs=0, epsrel=1e-13, limit=400)[0]
    outer = integrate.quad(lambda s: rho_of_r(s) * s, min(r, R), R, epsabs=0, epsrel=1e-13, limit=400)[0] \
        if r < R else 0.0
    if r == 0.0:
        return integrate.quad(lambda s: rho_of_r(s) * s, 0.0, R, epsabs=0, epsrel=1e-13, limit=400)[0]
    return inner / r + outer


def rel_err(u, ue):
    """E of eq. (error_infty): max |u - u*| / max |u*|."""
    return float(np.abs(u - ue).max() / np.abs(ue).max())


def read_table(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(tuple(float(t) for t in line.split()))
    return rows
