"""ctypes binding of ``libsuperpot.so`` (the C ABI of include/superpot.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Importing this module loads the library and raises ``ImportError``
when it has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsuperpot.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "superpot.h")

SP_FP64, SP_FP32, SP_MIXED = 0, 1, 2
STATUS = {0: "SP_OK", 1: "SP_ERR_INVALID", 2: "SP_ERR_UNSUPPORTED_SIZE", 3: "SP_ERR_OOM",
          4: "SP_ERR_CUDA", 5: "SP_ERR_TIMEOUT", 6: "SP_ERR_NOT_READY"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(the solver has no CPU fallback)")

lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

lib.sp_plan_create.restype = ctypes.c_int
lib.sp_plan_create.argtypes = [ctypes.POINTER(_vp), _ip, _dp, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int,
                               ctypes.c_double, ctypes.c_int, ctypes.c_int]
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    """sp_allocator of include/superpot.h."""
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", ctypes.c_void_p)]


lib.sp_plan_create_ex.restype = ctypes.c_int
lib.sp_plan_create_ex.argtypes = [ctypes.POINTER(_vp), _ip, _dp, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Allocator)]
lib.sp_solve_host.restype = ctypes.c_int
lib.sp_solve_host.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, _vp]
lib.sp_plan_set_persistent.restype = ctypes.c_int
lib.sp_plan_set_persistent.argtypes = [_vp, ctypes.c_int]
lib.sp_plan_barrier_check.restype = ctypes.c_int
lib.sp_plan_barrier_check.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _vp]
class ServerConfig(ctypes.Structure):
    """sp_server_config of include/superpot.h."""
    _fields_ = [("lo", ctypes.c_double), ("hi", ctypes.c_double), ("budget_bytes", ctypes.c_double),
                ("max_batch", ctypes.c_int), ("slots", ctypes.c_int), ("priority_slots", ctypes.c_int),
                ("plans_per_key", ctypes.c_int), ("small_points", ctypes.c_longlong),
                ("max_batch_points", ctypes.c_longlong)]


class ServerRecord(ctypes.Structure):
    """sp_server_record of include/superpot.h."""
    _fields_ = [("arrival", ctypes.c_double), ("launched", ctypes.c_double), ("done", ctypes.c_double),
                ("n", ctypes.c_int), ("precision", ctypes.c_int)]


_llp = ctypes.POINTER(ctypes.c_longlong)
lib.sp_server_create.restype = ctypes.c_int
lib.sp_server_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(ServerConfig)]
lib.sp_server_prepare.restype = ctypes.c_int
lib.sp_server_prepare.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
lib.sp_server_submit.restype = ctypes.c_int
lib.sp_server_submit.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_double, _llp]
lib.sp_server_replay.restype = ctypes.c_int
lib.sp_server_replay.argtypes = [_vp, ctypes.c_int, _dp, _ip, _ip, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _llp]
lib.sp_server_next_done.restype = ctypes.c_int
lib.sp_server_next_done.argtypes = [_vp, ctypes.c_double, _llp, _dp]
lib.sp_server_stats.restype = ctypes.c_int
lib.sp_server_stats.argtypes = [_vp, _llp, _dp, _dp]
lib.sp_server_records.restype = ctypes.c_int
lib.sp_server_records.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ServerRecord)]
lib.sp_server_shutdown.restype = ctypes.c_int
lib.sp_server_shutdown.argtypes = [_vp]
lib.sp_server_destroy.restype = ctypes.c_int
lib.sp_server_destroy.argtypes = [_vp]
lib.sp_server_entry_bytes.restype = ctypes.c_size_t
lib.sp_server_entry_bytes.argtypes = [ctypes.POINTER(ServerConfig), ctypes.c_int, ctypes.c_int]
lib.sp_monotonic_seconds.restype = ctypes.c_double
lib.sp_monotonic_seconds.argtypes = []
lib.sp_plan_sync.restype = ctypes.c_int
lib.sp_plan_sync.argtypes = [_vp]
lib.sp_kernel_precompute.restype = ctypes.c_int
lib.sp_kernel_precompute.argtypes = [_vp, _vp]
lib.sp_solve.restype = ctypes.c_int
lib.sp_solve.argtypes = [_vp, _vp, _vp, _vp]
lib.sp_solve_batched.restype = ctypes.c_int
lib.sp_solve_batched.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp]
lib.sp_forward_spectrum.restype = ctypes.c_int
lib.sp_forward_spectrum.argtypes = [_vp, _vp, _vp, _vp]
lib.sp_plan_destroy.restype = ctypes.c_int
lib.sp_plan_destroy.argtypes = [_vp]
lib.sp_plan_workspace_bytes.restype = ctypes.c_size_t
lib.sp_plan_workspace_bytes.argtypes = [_vp]
lib.sp_plan_gs_terms.restype = ctypes.c_int
lib.sp_plan_gs_terms.argtypes = [_vp]
lib.sp_plan_copy_tables.restype = ctypes.c_int
lib.sp_plan_copy_tables.argtypes = [_vp, _dp, _dp, _dp, ctypes.c_int, _dp, _dp]
lib.sp_bluestein_table.restype = ctypes.c_int
lib.sp_bluestein_table.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _vp, ctypes.POINTER(ctypes.c_size_t)]
lib.sp_plan_set_timing.restype = ctypes.c_int
lib.sp_plan_set_timing.argtypes = [_vp, ctypes.c_int]
lib.sp_plan_pass_times.restype = ctypes.c_int
lib.sp_plan_pass_times.argtypes = [_vp, _dp, _ip, ctypes.POINTER(ctypes.c_char_p), ctypes.c_int]
lib.sp_plan_set_kernel.restype = ctypes.c_int
lib.sp_plan_set_kernel.argtypes = [_vp, ctypes.c_int]
lib.sp_plan_autotune.restype = ctypes.c_int
lib.sp_plan_autotune.argtypes = [_vp, ctypes.c_int, _vp]
lib.sp_plan_launch_config.restype = ctypes.c_int
lib.sp_plan_launch_config.argtypes = [_vp, _ip, _ip, _ip, _ip, _ip]
lib.sp_plan_set_launch_config.restype = ctypes.c_int
lib.sp_plan_set_launch_config.argtypes = [_vp, _ip, ctypes.c_int, _ip, ctypes.c_int]
lib.sp_plan_tiles.restype = ctypes.c_int
lib.sp_plan_tiles.argtypes = [_vp, _ip, _ip]
lib.sp_graph_capture.restype = ctypes.c_int
lib.sp_graph_capture.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.POINTER(_vp)]
lib.sp_graph_launch.restype = ctypes.c_int
lib.sp_graph_launch.argtypes = [_vp, _vp]
lib.sp_graph_destroy.restype = ctypes.c_int
lib.sp_graph_destroy.argtypes = [_vp]
lib.sp_solve_noalloc.restype = ctypes.c_int
lib.sp_solve_noalloc.argtypes = [_vp, _vp, _vp, _vp]
lib.sp_last_error.restype = ctypes.c_char_p
lib.sp_last_error.argtypes = []
lib.sp_version.restype = ctypes.c_char_p
lib.sp_version.argtypes = []


class SuperpotError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        self.status = STATUS.get(code, str(code))
        msg = lib.sp_last_error().decode(errors="replace")
        super().__init__(f"{where}: {self.status}: {msg}")


def check(code: int, where: str) -> None:
    if code != 0:
        raise SuperpotError(code, where)


def declared_symbols(header: str = HEADER):
    """Names of the functions declared in the public header."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sp_[a-z_0-9]+)\s*\(", text)))
