"""Seeded synthetic densities on uniform grids.

This module only samples source densities; it holds none of the solver's
arithmetic and is shared by the CUDA path's tests and the oracle's tests as the
common input generator.  Every density is one the paper (or the benchmark
configurations built on it) uses:

* ``gaussian``        normalised Gaussian, eq. (gaussian) of Sec. 3.1
* ``two_gaussians``   superposed Gaussians, eq. (gaussians) of Sec. 3.1
* ``paper_bump``      the bump density of eq. (bump), Sec. 3.2
* ``anisotropic``     eq. (anis), Sec. 3.3
* ``oscillating``     eq. (osci), Sec. 3.4
* ``bump_profile``    exp(-1/(1 - r^2/R^2)) on r < R (the C-infinity bump used
                      as a density in the large-grid workloads)
* ``cos_gaussian``    exp(-r^2/(2 s^2)) cos(w x) cos(w y) cos(w z)
* ``gaussian_mixture`` seeded mixture of 1..8 normalised Gaussians

The grid is x_j = lo + j (hi - lo)/(n - 1) per axis (both faces are grid
points), arrays are C-order ``[x][y][z]`` float64.
"""
from __future__ import annotations

import math

import numpy as np


def _vec3(v):
    if np.isscalar(v):
        return (v, v, v)
    v = tuple(v)
    assert len(v) == 3
    return v


def axes(n, lo, hi):
    """Coordinates of the grid points along each axis."""
    n, lo, hi = _vec3(n), _vec3(lo), _vec3(hi)
    return [float(a) + (float(b) - float(a)) / (int(m) - 1) * np.arange(int(m), dtype=np.float64)
            for m, a, b in zip(n, lo, hi)]


def mesh(n, lo, hi):
    x, y, z = axes(n, lo, hi)
    return np.meshgrid(x, y, z, indexing="ij")


def _r2(n, lo, hi, c):
    X, Y, Z = mesh(n, lo, hi)
    c = _vec3(c)
    return (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2


def gaussian(n, lo, hi, sigma, c=(0.0, 0.0, 0.0)):
    r2 = _r2(n, lo, hi, c)
    return np.exp(-r2 / (2.0 * sigma * sigma)) / ((2.0 * math.pi) ** 1.5 * sigma ** 3)


def two_gaussians(n, lo, hi, sigma1, sigma2, c, d):
    c, d = np.asarray(_vec3(c), float), np.asarray(_vec3(d), float)
    return 0.5 * (gaussian(n, lo, hi, sigma1, c + d) + gaussian(n, lo, hi, sigma2, c - d))


def paper_bump(n, lo, hi, R, d, c=(0.0, 0.0, 0.0)):
    """-Laplacian of u*(x) = exp(-d/(1 - |x-c|^2/R^2)) on |x-c| < R, else 0.

    The printed eq. (bump) differs from -Laplacian(u*) (its r^2 coefficient and
    its exponent); the density used here is the exact -Laplacian of the stated
    exact solution:
        2 d R^2 (3R^4 - 2R^2 r^2 - r^4 - 2 d R^2 r^2) / (R^2 - r^2)^4 * exp(-d R^2/(R^2 - r^2)).
    """
    r2 = _r2(n, lo, hi, c)
    R2 = R * R
    out = np.zeros_like(r2)
    m = r2 < R2
    q = r2[m]
    num = 3 * R2 * R2 - 2 * R2 * q - q * q - 2 * d * R2 * q
    out[m] = 2 * d * R2 * num / (R2 - q) ** 4 * np.exp(-d * R2 / (R2 - q))
    return out


def anisotropic(n, lo, hi, sig, c=(0.0, 0.0, 0.0)):
    X, Y, Z = mesh(n, lo, hi)
    sx, sy, sz = _vec3(sig)
    cx, cy, cz = _vec3(c)
    dx, dy, dz = X - cx, Y - cy, Z - cz
    e = np.exp(-dx * dx / sx ** 2 - dy * dy / sy ** 2 - dz * dz / sz ** 2)
    poly = 4 * dx * dx / sx ** 4 + 4 * dy * dy / sy ** 4 + 4 * dz * dz / sz ** 4 \
        - 2 / sx ** 2 - 2 / sy ** 2 - 2 / sz ** 2
    return -poly * e


def oscillating(n, lo, hi, sigma, omega, c=(0.0, 0.0, 0.0)):
    """-Laplacian of u*(x) = exp(-r^2/sigma^2) cos(omega r^2), r = |x - c|.

    The printed eq. (osci) carries -4 omega^2 r^2 cos(omega r^2) inside its first
    bracket; the exact -Laplacian of the stated solution has +4 omega^2 r^2, which
    is used here.
    """
    r2 = _r2(n, lo, hi, c)
    e = np.exp(-r2 / sigma ** 2)
    s, co = np.sin(omega * r2), np.cos(omega * r2)
    return (e * (6 * omega * s + 4 * omega ** 2 * r2 * co)
            - (4 * r2 / sigma ** 4 - 6 / sigma ** 2) * e * co
            - 8 * omega * r2 / sigma ** 2 * e * s)


def bump_profile(n, lo, hi, R=0.8, c=(0.0, 0.0, 0.0)):
    r2 = _r2(n, lo, hi, c)
    out = np.zeros_like(r2)
    m = r2 < R * R
    out[m] = np.exp(-1.0 / (1.0 - r2[m] / (R * R)))
    return out


def cos_gaussian(n, lo, hi, s=0.25, w=8.0 * math.pi):
    X, Y, Z = mesh(n, lo, hi)
    return np.exp(-(X * X + Y * Y + Z * Z) / (2 * s * s)) * np.cos(w * X) * np.cos(w * Y) * np.cos(w * Z)


def mixture_params(seed: int):
    """Seeded mixture parameters: K ~ U{1..8}, centres U[-0.5,0.5]^3,
    sigma ~ U[0.05, 0.2], weights ~ U[-1, 1] (numpy PCG64)."""
    g = np.random.Generator(np.random.PCG64(seed))
    K = int(g.integers(1, 9))
    centres = g.uniform(-0.5, 0.5, size=(K, 3))
    sig = g.uniform(0.05, 0.2, size=K)
    wts = g.uniform(-1.0, 1.0, size=K)
    return centres, sig, wts


def gaussian_mixture(n, lo, hi, seed: int):
    centres, sig, wts = mixture_params(seed)
    out = np.zeros(tuple(_vec3(n)))
    for c, s, w in zip(centres, sig, wts):
        out += w * gaussian(n, lo, hi, s, c)
    return out
