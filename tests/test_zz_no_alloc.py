"""sp_solve_noalloc, the solve for callers that cannot allocate device memory.

Some programs must not allocate at the moment they solve: cudaMalloc/cudaFree can
synchronise the whole device and stall a latency-bound time loop, a host framework
may keep all device memory in its own pool, or the memory budget is fixed at start-up.
For them the library offers sp_solve_noalloc, which runs the same passes as sp_solve
but keeps its workspace in a static device array compiled into the library.

This file calls it through the C ABI, twice in a row with different densities (so
the second call cannot lean on what the first left in the shared array), and checks
each result against sp_solve's within the parity tolerances used elsewhere (FP64
1e-12, FP32 1e-5, max-norm relative).  It is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "df32": 1e-12, "fp32": 1e-5, "mixed": 1e-5}


def _noalloc(native, plan, rho, u):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return native.lib.sp_solve_noalloc(plan.handle, ctypes.c_void_p(rho.data_ptr()),
                                       ctypes.c_void_p(u.data_ptr()), stream)


@pytest.mark.parametrize("precision,n", [("fp64", (48, 64, 36)), ("fp64", (96, 96, 96)),
                                         ("fp32", (128, 128, 128)), ("mixed", (64, 64, 64)),
                                         ("df32", (64, 96, 64))])
def test_noalloc_matches_solve_twice(precision, n):
    from paper_2506_04489_gb300 import Plan, _native, workloads as W
    plan = Plan(n, (-1.0, -1.2, -0.8), (1.0, 1.2, 0.9), precision=precision)
    for seed in (5, 6):
        rho = torch.from_numpy(W.gaussian_mixture(n, (-1.0, -1.2, -0.8), (1.0, 1.2, 0.9), seed)).cuda()
        rho = rho.to(plan.dtype)
        ref = plan.solve(rho)
        u = torch.full_like(rho, float("nan"))
        rc = _noalloc(_native, plan, rho, u)
        assert rc == 0, _native.lib.sp_last_error()
        torch.cuda.synchronize()
        err = float((u.double() - ref.double()).abs().max() / ref.double().abs().max())
        assert err <= TOL[precision], (seed, err)
    plan.close()


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    from paper_2506_04489_gb300 import Plan, _native
    plan = Plan(128, -1.0, 1.0, precision="fp64")  # 71 MB of workspace > 64 MiB
    rho = torch.zeros((128, 128, 128), dtype=torch.float64, device="cuda")
    u = torch.empty_like(rho)
    assert _noalloc(_native, plan, rho, u) == 2  # SP_ERR_UNSUPPORTED_SIZE
    assert b"static scratch" in _native.lib.sp_last_error()
    plan.close()
