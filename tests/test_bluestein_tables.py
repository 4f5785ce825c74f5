"""Host-built tables of Bluestein's algorithm (sp_bluestein_table; no GPU): the chirp and
the filter spectra a plan uses on axes whose padded length 2n has a prime factor above 7.

Independent references: numpy's FFT of the filter, and the whole chirp-z transform run
in numpy with the returned tables against numpy.fft of the same line (the tables must
turn a length-N DFT into the M-point convolution they are built for, in both
directions).
"""
import ctypes

import numpy as np
import pytest

PREC = {"fp64": 0, "fp32": 1, "mixed": 2, "df32": 3}
# per value: (complex value tolerance of the stored tables, transform tolerance / sum|x|)
TOL = {"fp64": (2e-15, 1e-13), "df32": (2e-14, 1e-12), "fp32": (2e-7, 2e-5), "mixed": (2e-7, 2e-5)}


@pytest.fixture(scope="module")
def native():
    from paper_2506_04489_gb300 import build
    build.build()
    from paper_2506_04489_gb300 import _native
    return _native


def _table(native, n, prec):
    M, nbytes = ctypes.c_int(), ctypes.c_size_t(0)
    rc = native.lib.sp_bluestein_table(n, PREC[prec], ctypes.byref(M), None, ctypes.byref(nbytes))
    assert rc == 0, native.lib.sp_last_error()
    buf = (ctypes.c_ubyte * nbytes.value)()
    rc = native.lib.sp_bluestein_table(n, PREC[prec], ctypes.byref(M), buf, ctypes.byref(nbytes))
    assert rc == 0, native.lib.sp_last_error()
    raw = np.frombuffer(bytes(buf), dtype=np.float64 if prec == "fp64" else np.float32)
    if prec == "fp64":
        vals = raw[0::2] + 1j * raw[1::2]
    elif prec == "df32":  # re.hi, im.hi, re.lo, im.lo
        r = raw.reshape(-1, 4).astype(np.float64)
        vals = (r[:, 0] + r[:, 2]) + 1j * (r[:, 1] + r[:, 3])
    else:
        vals = raw[0::2].astype(np.float64) + 1j * raw[1::2].astype(np.float64)
    return M.value, nbytes.value, vals


@pytest.mark.parametrize("n", [11, 13, 61, 101, 1021])
@pytest.mark.parametrize("prec", ["fp64", "df32", "fp32", "mixed"])
def test_tables_and_the_transform_they_give(native, n, prec):
    N = 2 * n
    M, nbytes, t = _table(native, n, prec)
    assert M >= 2 * N - 1 and M & (M - 1) == 0 and M < 2 * (2 * N - 1)
    assert nbytes == (16 if prec in ("fp64", "df32") else 8) * (N + 3 * M)
    chirp, dfwd, dinv, tw = t[:N], t[N:N + M], t[N + M:N + 2 * M], t[N + 2 * M:]
    tol_v, tol_x = TOL[prec]
    j = np.arange(N)
    c = np.exp(-1j * np.pi * ((j * j) % (2 * N)) / N)
    assert np.abs(chirp - c).max() <= tol_v
    for got, f in ((dfwd, np.conj(c)), (dinv, c)):
        e = np.zeros(M, complex)
        e[:N] = f
        e[M - np.arange(1, N)] = f[1:]
        assert np.abs(got - np.fft.fft(e) / M).max() <= 4 * tol_v
    q = np.arange(M)
    assert np.abs(tw - np.exp(-2j * np.pi * q / M)).max() <= tol_v
    # the chirp-z transform with these tables, in numpy
    x = np.random.default_rng(n).standard_normal(N) + 1j * np.random.default_rng(n + 1).standard_normal(N)
    for sign, D in ((-1, dfwd), (+1, dinv)):
        ch = chirp if sign < 0 else np.conj(chirp)
        a = np.zeros(M, complex)
        a[:N] = x * ch
        conv = np.fft.ifft(np.fft.fft(a) * D) * M  # D carries the 1/M of the inverse
        X = conv[:N] * ch
        ref = np.fft.fft(x) if sign < 0 else N * np.fft.ifft(x)
        assert np.abs(X - ref).max() <= tol_x * np.abs(x).sum(), sign


@pytest.mark.parametrize("n,prec,code", [(8, "fp64", 2), (32, "df32", 2), (35, "fp32", 2), (1, "fp64", 2),
                                         (1025, "fp64", 2), (11, None, 1)])
def test_rejects_other_lengths_and_arguments(native, n, prec, code):
    M, nbytes = ctypes.c_int(), ctypes.c_size_t(0)
    p = 9 if prec is None else PREC[prec]
    assert native.lib.sp_bluestein_table(n, p, ctypes.byref(M), None, ctypes.byref(nbytes)) == code


def test_rejects_a_short_buffer(native):
    M, nbytes = ctypes.c_int(), ctypes.c_size_t(0)
    assert native.lib.sp_bluestein_table(11, 0, ctypes.byref(M), None, ctypes.byref(nbytes)) == 0
    small = ctypes.c_size_t(nbytes.value - 16)
    buf = (ctypes.c_ubyte * nbytes.value)()
    assert native.lib.sp_bluestein_table(11, 0, ctypes.byref(M), buf, ctypes.byref(small)) == 1
