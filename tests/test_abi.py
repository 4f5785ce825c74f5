"""C-ABI checks that need no GPU: the library loads, exports every function the
public header declares, and rejects invalid plans before touching the device."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def native():
    from paper_2506_04489_gb300 import build
    build.build()
    from paper_2506_04489_gb300 import _native
    return _native


def test_exports_every_declared_symbol(native):
    names = native.declared_symbols()
    assert "sp_plan_create" in names and "sp_solve" in names and "sp_kernel_precompute" in names
    for name in names:
        assert hasattr(native.lib, name), name


def _create(native, n=(8, 8, 8), lo=(-1,) * 3, hi=(1,) * 3, padding=2, gs=None, eps=1e-4, prec=0, mb=1):
    h = ctypes.c_void_p()
    nn = (ctypes.c_int * 3)(*n)
    l = (ctypes.c_double * 3)(*lo)
    u = (ctypes.c_double * 3)(*hi)
    if gs is None:
        w = a = None
        t = 0
    else:
        w = (ctypes.c_double * len(gs[0]))(*gs[0])
        a = (ctypes.c_double * len(gs[1]))(*gs[1])
        t = len(gs[0])
    rc = native.lib.sp_plan_create(ctypes.byref(h), nn, l, u, padding, w, a, t, eps, prec, mb)
    return rc, h


# any n >= 2 with 2n <= 2048 is accepted (lengths with a prime factor above 7 through
# Bluestein's algorithm); smaller or larger grids are refused before any allocation
@pytest.mark.parametrize("n,code", [((1, 8, 8), 2), ((8, 1, 8), 2), ((8, 8, 0), 2), ((8, 8, 2048), 2),
                                    ((1025, 8, 8), 2), ((8, 8, 1025), 2)])
def test_rejects_unsupported_sizes(native, n, code):
    rc, h = _create(native, n=n)
    assert rc == code and not h.value
    assert b"n[" in native.lib.sp_last_error()


# double-float takes the same lengths as the other precisions (register-resident passes
# where a plan is compiled, the first-generation passes elsewhere): the same rule rejects
@pytest.mark.parametrize("n", [(1, 8, 8), (8, 1, 8), (8, 8, 2048), (1025, 8, 8)])
def test_double_float_rejects_unsupported_sizes(native, n):
    rc, h = _create(native, n=n, prec=3)
    assert rc == 2 and not h.value
    assert b"n[" in native.lib.sp_last_error()


def test_rejects_invalid_arguments(native):
    assert _create(native, padding=3)[0] == 1
    assert _create(native, lo=(1, -1, -1), hi=(-1, 1, 1))[0] == 1
    assert _create(native, prec=7)[0] == 1
    assert _create(native, mb=0)[0] == 1
    assert _create(native, eps=0.0)[0] == 1
    assert _create(native, gs=([1.0, 2.0], [1.0, -1.0]))[0] == 1
    assert native.lib.sp_solve(None, None, None, None) == 1
    assert native.lib.sp_plan_destroy(None) == 0
    assert native.lib.sp_plan_workspace_bytes(None) == 0


def test_new_entry_points_reject_invalid_arguments(native):
    # allocator without callbacks: refused before any device memory is touched
    h = ctypes.c_void_p()
    nn = (ctypes.c_int * 3)(8, 8, 8)
    lo = (ctypes.c_double * 3)(-1, -1, -1)
    hi = (ctypes.c_double * 3)(1, 1, 1)
    bad = native.Allocator()
    assert native.lib.sp_plan_create_ex(ctypes.byref(h), nn, lo, hi, 2, None, None, 0, 1e-4, 0, 1,
                                        ctypes.byref(bad)) == 1
    assert not h.value and b"allocator" in native.lib.sp_last_error()
    assert native.lib.sp_plan_sync(None) == 1
    assert native.lib.sp_solve_host(None, None, None, 1, None) == 1
