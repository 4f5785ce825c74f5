"""Batched solves (many right-hand sides of one size): tile autotuning, CUDA-graph
capture and replay, and the rule that a result in the batch equals the same solve alone.

Workload: 64 right-hand sides on a 128^3 grid of [-1,1]^3, each a seeded mixture of
1-8 normalised Gaussians (seed = index), solved in one batched call replayed from a
captured graph.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan, workloads as W  # noqa: E402

N, LO, HI, BATCH = 128, -1.0, 1.0, 64
TOL = {"fp64": 1e-12, "df32": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def rhs():
    return torch.stack([torch.from_numpy(W.gaussian_mixture(N, LO, HI, s)) for s in range(BATCH)])


@pytest.mark.parametrize("precision", ["df32", "fp32", "fp64"])
def test_batched_graph_matches_alone_and_oracle(oracle, rhs, precision):
    plan = Plan(N, LO, HI, precision=precision, max_batch=BATCH)
    rho = rhs.to("cuda", dtype=plan.dtype)
    tiles = plan.autotune(BATCH)
    assert tiles["z"] > 0 and tiles["line"][0] > 0 and tiles["line"][1] > 0
    # reference: every right-hand side alone, in the same launch configuration (the tuner
    # may have picked another radix plan, which rounds differently)
    alone = torch.stack([plan.solve(rho[b].contiguous()) for b in range(BATCH)])
    out = torch.empty_like(rho)
    stream = torch.cuda.Stream()
    # the plan's solves share one workspace: the capture's solves on `stream` must follow
    # the ones above on the current stream
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        graph = plan.capture(rho, out, stream)
        out.zero_()
        graph.launch(stream)
    stream.synchronize()
    # same kernels per right-hand side, tiles do not change the arithmetic: bitwise equal
    assert torch.equal(out, alone)
    # replay after changing the inputs in place (the copy is ordered on the same stream)
    rho2 = torch.flip(rho, dims=[1]).contiguous()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        rho.copy_(rho2)
        graph.launch(stream)
    stream.synchronize()
    for b in (0, 17):
        assert torch.equal(out[b], plan.solve(rho[b].contiguous()))
    graph.close()
    # a sample against the oracle
    _, _, M = oracle.plan_tables(N, LO, HI)
    for b in (3, 40):
        ref = oracle.solve(M, rho[b].double().cpu().numpy())
        got = out[b].double().cpu().numpy()
        assert np.abs(got - ref).max() / np.abs(ref).max() <= TOL[precision]
    plan.close()


def test_autotune_keeps_results_bitwise(oracle):
    plan = Plan((64, 96, 64), (-1, -1.5, -1), (1, 1.5, 1), precision="fp32", max_batch=2)
    rho = torch.from_numpy(np.stack([W.gaussian_mixture((64, 96, 64), (-1, -1.5, -1), (1, 1.5, 1), s)
                                     for s in (1, 2)])).float().cuda()
    before = plan.solve_batched(rho)
    plan.autotune(2)
    after = plan.solve_batched(rho)
    assert torch.equal(before, after)
    plan.close()


@pytest.mark.parametrize("precision", ["df32", "fp32"])
def test_host_stream_matches_device_solves(rhs, precision):
    # overlapped host->device->host solves give the same bits as device-resident solves,
    # for a sequence longer than the two staging buffers and with repeated host buffers
    plan = Plan(N, LO, HI, precision=precision)
    k = 7
    ins = [rhs[b].to(dtype=plan.dtype).pin_memory() for b in range(k)]
    outs = [torch.empty_like(x).pin_memory() for x in ins]
    plan.solve_host_stream(ins, outs)
    for b in range(k):
        want = plan.solve(ins[b].cuda()).cpu()
        assert torch.equal(outs[b], want), b
    # one input buffer reused for every step, fresh outputs
    outs2 = [torch.empty_like(ins[0]).pin_memory() for _ in range(3)]
    plan.solve_host_stream([ins[2]] * 3, outs2)
    for o in outs2:
        assert torch.equal(o, outs[2])
    # wrong dtype, wrong shape, device tensors and unequal lengths are rejected
    other = torch.float64 if plan.dtype == torch.float32 else torch.float32
    with pytest.raises(ValueError):
        plan.solve_host_stream([ins[0].to(other)], [outs[0]])
    with pytest.raises(ValueError):
        plan.solve_host_stream([ins[0][:-1]], [outs[0]])
    with pytest.raises(ValueError):
        plan.solve_host_stream([ins[0].cuda()], [outs[0]])
    with pytest.raises(ValueError):
        plan.solve_host_stream(ins[:2], outs[:1])
    plan.close()
