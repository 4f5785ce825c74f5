"""The persistent solve: all five passes of Alg. 2 in one cooperative launch with grid
barriers between them (the batched configuration's single fused launch), and the bounded
wait of its barrier.

Tiles only regroup lines into CTAs, so the persistent launch must reproduce the five-launch
solve bit for bit, alone, batched and replayed from a captured graph; one case also meets
the oracle directly.  The barrier's wait gives up after its limit and reports it through
sp_plan_sync (SP_ERR_TIMEOUT), which the test provokes with a barrier that waits for one
block more than were launched; the context stays usable afterwards.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan, workloads as W  # noqa: E402
from paper_2506_04489_gb300._native import SuperpotError  # noqa: E402


def _batch(n, nb, dtype):
    return torch.stack([torch.from_numpy(W.gaussian_mixture(n, -1.0, 1.0, s)) for s in range(nb)]).to("cuda", dtype)


@pytest.mark.parametrize("n", [32, 64, 96, 128, 192, 256])
@pytest.mark.parametrize("precision", ["df32", "fp32", "mixed", "fp64"])
def test_persistent_equals_five_launches(n, precision):
    nb = 3 if n <= 128 else 1
    plan = Plan(n, -1.0, 1.0, precision=precision, max_batch=nb)
    rhos = _batch(n, nb, plan.dtype)
    ref = plan.solve_batched(rhos)
    plan.set_persistent(True)
    got = plan.solve_batched(rhos)
    plan.sync()
    assert torch.equal(got, ref)
    assert torch.equal(plan.solve(rhos[0].contiguous()), ref[0])
    st = torch.cuda.Stream()
    out = torch.full_like(rhos, float("nan"))
    graph = plan.capture(rhos, out, st)
    out.fill_(float("nan"))
    graph.launch(st)
    st.synchronize()
    plan.sync()
    assert torch.equal(out, ref)
    graph.close()
    plan.close()


def test_persistent_matches_oracle(oracle):
    n = 64
    rho = W.gaussian_mixture(n, -1.0, 1.0, 9) + 0.01 * np.random.default_rng(9).standard_normal((n, n, n))
    _, _, M = oracle.plan_tables(n, -1.0, 1.0)
    ref = oracle.solve(M, rho)
    plan = Plan(n, -1.0, 1.0, precision="df32")
    plan.set_persistent(True)
    u = plan.solve(torch.from_numpy(rho).cuda()).cpu().numpy()
    plan.sync()
    plan.close()
    assert np.abs(u - ref).max() / np.abs(ref).max() <= 1e-12


def test_persistent_needs_a_cubic_compiled_grid():
    plan = Plan((64, 32, 64), -1.0, 1.0, precision="df32")
    with pytest.raises(SuperpotError) as e:
        plan.set_persistent(True)
    assert e.value.status == "SP_ERR_UNSUPPORTED_SIZE"
    plan.close()


def test_barrier_wait_is_bounded_and_reported():
    plan = Plan(32, -1.0, 1.0, precision="df32")
    rho = torch.from_numpy(W.gaussian(32, -1.0, 1.0, 0.2)).cuda()
    before = plan.solve(rho)
    plan.barrier_check(4, 4, 50.0)  # every arrival comes: the barrier completes
    plan.sync()
    t0 = time.perf_counter()
    plan.barrier_check(2, 3, 50.0)  # waits for a block that was never launched
    with pytest.raises(SuperpotError) as e:
        plan.sync()
    assert e.value.status == "SP_ERR_TIMEOUT"
    assert time.perf_counter() - t0 < 10.0
    plan.sync()  # the status word was cleared
    # the context is usable: solves still run and agree
    assert torch.equal(plan.solve(rho), before)
    plan.sync()
    plan.close()
