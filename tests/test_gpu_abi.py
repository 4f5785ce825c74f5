"""Boundary behaviour on the GPU: the plan's completion event (destroy and sp_plan_sync
wait for the plan's own work), plan memory from the caller's allocator, and the
host-buffer entry sp_solve_host against device solves."""
import ctypes
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan, workloads as W  # noqa: E402


def test_sync_reports_ok_and_waits_for_the_plan():
    plan = Plan(64, -1.0, 1.0, precision="df32")
    rho = torch.from_numpy(W.gaussian_mixture(64, -1.0, 1.0, 1)).cuda()
    u = plan.solve(rho)
    plan.sync()  # SP_OK: nothing timed out, no device error
    ref = plan.solve(rho.clone())
    plan.sync()
    assert torch.equal(u, ref)
    plan.close()


def test_destroy_waits_for_own_work_not_the_device():
    # Another stream keeps the device busy for a while; destroying a plan whose work is
    # done must not wait for it (the old behaviour synchronised the whole device).
    side = torch.cuda.Stream()
    big = torch.empty(2 ** 28, dtype=torch.float32, device="cuda")
    plan = Plan(32, -1.0, 1.0, precision="fp64")
    rho = torch.from_numpy(W.gaussian(32, -1.0, 1.0, 0.2)).cuda()
    plan.solve(rho)
    plan.sync()
    with torch.cuda.stream(side):
        for _ in range(200):
            big.mul_(1.0000001)  # ~200 passes over 1 GB: tens of milliseconds of work
    t0 = time.perf_counter()
    plan.close()
    closed = time.perf_counter() - t0
    t1 = time.perf_counter()
    side.synchronize()
    rest = time.perf_counter() - t1
    assert closed < rest, (closed, rest)


def test_torch_allocator_plan_matches_default():
    n = (48, 64, 40)
    rho = torch.from_numpy(W.gaussian_mixture(n, -1.0, 1.0, 2)).cuda()
    before = torch.cuda.memory_allocated()
    p_t = Plan(n, -1.0, 1.0, precision="fp64", allocator="torch")
    held = torch.cuda.memory_allocated() - before
    assert held >= p_t.workspace_bytes  # the plan's memory came from torch's pool
    p_d = Plan(n, -1.0, 1.0, precision="fp64")
    assert torch.equal(p_t.solve(rho), p_d.solve(rho))
    p_t.close()
    p_d.close()
    assert torch.cuda.memory_allocated() == before  # released through the allocator


@pytest.mark.parametrize("precision", ["df32", "fp32"])
def test_solve_host_matches_device_solves(precision):
    n = (64, 32, 96)
    plan = Plan(n, -1.0, 1.0, precision=precision)
    dt = plan.dtype
    ins = [torch.from_numpy(W.gaussian_mixture(n, -1.0, 1.0, s)).to(dt).pin_memory() for s in range(5)]
    outs = [torch.empty(n, dtype=dt).pin_memory() for _ in range(5)]
    plan.solve_host_stream(ins, outs)
    for x, y in zip(ins, outs):
        assert torch.equal(plan.solve(x.cuda()).cpu(), y)
    # a second call reuses the staging buffers; one array in and out in place
    x = ins[2].clone().pin_memory()
    plan.solve_host_stream([x], [x])
    assert torch.equal(x, outs[2])
    plan.close()
