"""Plain FP64 CPU oracle for the super-potential GS/FFT Poisson solve (arXiv:2506.04489).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method that the CUDA library is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  The product package never imports it, and it imports nothing
from the product package: the two share no code.

The arithmetic lives in ``sp_oracle.c`` (plain C, FP64, own FFT, adaptive
Gauss-Kronrod); this module only marshals numpy arrays through ctypes and
states the plan geometry:

* grid ``x_j = lo + j h`` with ``h = (hi - lo)/(n - 1)`` per axis (reading of
  Sec. 3, "mesh sizes h"; reproduces Tab. 1);
* padding factor 2 (Sec. 2, Alg. 1): window half-width ``L = n h``;
* GS range ``(eps, delta]`` with ``delta`` the window diagonal ``|L|`` (Thm. 1
  needs the GS accurate on every |y| of the window).

Parity pins for every function are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sp_oracle.c")
_LIB = os.path.join(_HERE, "libsp_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile ``sp_oracle.c`` into ``libsp_oracle.so`` beside it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.or_gs_table.restype = ctypes.c_int
            L.or_gs_table.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, _dp, _dp]
            L.or_gs_ratio.restype = ctypes.c_double
            L.or_gs_ratio.argtypes = [ctypes.c_double, ctypes.c_int, _dp, _dp]
            L.or_integrals_1d.restype = None
            L.or_integrals_1d.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp]
            L.or_axis_tables.restype = None
            L.or_axis_tables.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
            L.or_multiplier.restype = ctypes.c_int
            L.or_multiplier.argtypes = [_ip, _dp, ctypes.c_int, _dp, _dp, _dp]
            L.or_multiplier_gs_plain.restype = ctypes.c_int
            L.or_multiplier_gs_plain.argtypes = [_ip, _dp, ctypes.c_int, _dp, _dp, _dp]
            L.or_fft.restype = ctypes.c_int
            L.or_fft.argtypes = [ctypes.c_int, _dp, ctypes.c_int]
            L.or_fft3.restype = ctypes.c_int
            L.or_fft3.argtypes = [_ip, _dp, ctypes.c_int]
            L.or_solve.restype = ctypes.c_int
            L.or_solve.argtypes = [_ip, _dp, _dp, _dp]
            L.or_forward_spectrum.restype = ctypes.c_int
            L.or_forward_spectrum.argtypes = [_ip, _dp, _dp]
            L.or_dft_coeff.restype = ctypes.c_int
            L.or_dft_coeff.argtypes = [_ip, _dp, _ip, _dp, _dp]
            L.or_set_threads.restype = None
            L.or_set_threads.argtypes = [ctypes.c_int]
            L.or_get_threads.restype = ctypes.c_int
            L.or_get_threads.argtypes = []
            _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i3(v) -> ctypes.Array:
    return (ctypes.c_int * 3)(*[int(x) for x in v])


def set_threads(t: int) -> None:
    lib().or_set_threads(int(t))


def get_threads() -> int:
    return int(lib().or_get_threads())


# --------------------------------------------------------------------------- geometry
def _vec3(v):
    if np.isscalar(v):
        return (v, v, v)
    v = tuple(v)
    assert len(v) == 3
    return v


def geometry(n, lo, hi):
    """Per-axis (h, L): h = (hi-lo)/(n-1), L = n h (padding factor 2, Sec. 2)."""
    n, lo, hi = _vec3(n), _vec3(lo), _vec3(hi)
    h = tuple((float(b) - float(a)) / (int(m) - 1) for m, a, b in zip(n, lo, hi))
    L = tuple(int(m) * hh for m, hh in zip(n, h))
    return h, L


def default_delta(L) -> float:
    """Upper end of the GS range: the window diagonal (Thm. 1, the GS must cover B_2)."""
    return math.sqrt(sum(x * x for x in L))


# --------------------------------------------------------------------------- GS table
def gs_table(eps: float = 1e-4, delta: float = 2.0 * math.sqrt(3.0), h_tau: float = 0.1,
             eta: float = 1e-17):
    """(w_s, a_s) of eq. (sin_1_x) by sinc quadrature; see sp_oracle.c."""
    cap = 100000
    w = np.empty(cap)
    a = np.empty(cap)
    S1 = lib().or_gs_table(eps, delta, h_tau, eta, cap, _d(w), _d(a))
    if S1 < 0:
        raise ValueError("GS table too long")
    return w[:S1].copy(), a[:S1].copy()


def gs_ratio(r: float, w: np.ndarray, a: np.ndarray) -> float:
    """8 pi r U_GS(r) evaluated with a long-double accumulator (Fig. 1 quantity)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    return float(lib().or_gs_ratio(float(r), len(w), _d(w), _d(a)))


# --------------------------------------------------------------------------- 1D integrals
def integrals_1d(alpha: float, L: float, k: int):
    """(G, H) of eq. (Gten_sep) at kappa = pi k / L by adaptive Gauss-Kronrod."""
    G = ctypes.c_double()
    H = ctypes.c_double()
    lib().or_integrals_1d(float(alpha), float(L), int(k), ctypes.byref(G), ctypes.byref(H))
    return G.value, H.value


def axis_tables(n: int, L: float, a: np.ndarray):
    """G[s, k], H[s, k] for k = 0..n with kappa_k = pi k / L."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    G = np.empty((len(a), n + 1))
    H = np.empty((len(a), n + 1))
    lib().or_axis_tables(int(n), float(L), len(a), _d(a), _d(G), _d(H))
    return G, H


# --------------------------------------------------------------------------- multiplier
def multiplier(n, L, w: np.ndarray, a: np.ndarray) -> np.ndarray:
    """M[k0, k1, k2] = -|kappa|^2 Vhat_k for |k_p| = 0..n_p (eqs. convtheorem, Gten_sep)."""
    n = _vec3(n)
    L = _vec3(L)
    w = np.ascontiguousarray(w, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    M = np.empty((n[0] + 1, n[1] + 1, n[2] + 1))
    Lc = (ctypes.c_double * 3)(*[float(x) for x in L])
    if lib().or_multiplier(_i3(n), Lc, len(w), _d(w), _d(a), _d(M)) != 0:
        raise MemoryError("or_multiplier")
    return M


def multiplier_gs_plain(n, L, w: np.ndarray, a: np.ndarray) -> np.ndarray:
    """M[k] = sum_s 2 w_s G0 G1 G2: the original GS method without near-field correction."""
    n = _vec3(n)
    L = _vec3(L)
    w = np.ascontiguousarray(w, dtype=np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    M = np.empty((n[0] + 1, n[1] + 1, n[2] + 1))
    Lc = (ctypes.c_double * 3)(*[float(x) for x in L])
    if lib().or_multiplier_gs_plain(_i3(n), Lc, len(w), _d(w), _d(a), _d(M)) != 0:
        raise MemoryError("or_multiplier_gs_plain")
    return M


def plan_tables(n, lo, hi, eps: float = 1e-4, h_tau: float = 0.1, eta: float = 1e-17, kernel: str = "superpotential"):
    """GS table and multiplier for a box, with the default GS range (eps, |L|].
    kernel: "superpotential" (eq. convtheorem) or "gs_plain" (the original GS method
    without near-field correction)."""
    _, L = geometry(n, lo, hi)
    w, a = gs_table(eps, default_delta(L), h_tau, eta)
    if kernel == "gs_plain":
        return w, a, multiplier_gs_plain(_vec3(n), L, w, a)
    return w, a, multiplier(_vec3(n), L, w, a)


# --------------------------------------------------------------------------- FFT
def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised DFT of a 1D complex array, sum_j x_j exp(sign 2 pi i j k / m)."""
    buf = np.ascontiguousarray(x, dtype=np.complex128).copy()
    if lib().or_fft(len(buf), buf.view(np.float64).ctypes.data_as(_dp), int(sign)) != 0:
        raise MemoryError("or_fft")
    return buf


def fft3(x: np.ndarray, sign: int = -1) -> np.ndarray:
    buf = np.ascontiguousarray(x, dtype=np.complex128).copy()
    if lib().or_fft3(_i3(buf.shape), buf.view(np.float64).ctypes.data_as(_dp), int(sign)) != 0:
        raise MemoryError("or_fft3")
    return buf


# --------------------------------------------------------------------------- solve
def solve(M: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """u = crop(IDFT3(M .* DFT3(pad(rho))) / Ntilde)  (Alg. 2)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    n = rho.shape
    assert M.shape == tuple(m + 1 for m in n)
    M = np.ascontiguousarray(M, dtype=np.float64)
    u = np.empty_like(rho)
    if lib().or_solve(_i3(n), _d(M), _d(rho), _d(u)) != 0:
        raise MemoryError("or_solve")
    return u


def forward_spectrum(rho: np.ndarray) -> np.ndarray:
    """Padded forward DFT, half spectrum [2n0, 2n1, n2+1] (step 1 of Alg. 2)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    n = rho.shape
    S = np.empty((2 * n[0], 2 * n[1], n[2] + 1), dtype=np.complex128)
    if lib().or_forward_spectrum(_i3(n), _d(rho), S.view(np.float64).ctypes.data_as(_dp)) != 0:
        raise MemoryError("or_forward_spectrum")
    return S


def dft_coeff(rho: np.ndarray, k) -> complex:
    """One padded forward DFT coefficient by direct summation."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    re = ctypes.c_double()
    im = ctypes.c_double()
    if lib().or_dft_coeff(_i3(rho.shape), _d(rho), _i3(k), ctypes.byref(re), ctypes.byref(im)) != 0:
        raise MemoryError("or_dft_coeff")
    return complex(re.value, im.value)
