"""Grids off the register engine's compiled lengths (radix-5/7 lengths and Bluestein
lengths, with a prime factor above 7) through every entry point of the solve: batched
solves, a captured graph replayed, host-resident inputs and outputs.  Each result equals
the same right-hand side solved alone bit for bit (the same kernels per right-hand side),
and a sample meets the oracle at the parity tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan, workloads as W  # noqa: E402

TOL = {"fp64": 1e-12, "df32": 1e-12, "fp32": 1e-5, "mixed": 1e-5}
GRIDS = [(11, 13, 17), (20, 14, 25), (22, 16, 61)]  # 2n = 22, 26, 34 / 40, 28, 50 / 44, 32, 122
LO, HI = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)


def _rhs(n, count):
    rng = np.random.default_rng(sum(n))
    return [rng.standard_normal(n) for _ in range(count)]


@pytest.mark.parametrize("n", GRIDS)
@pytest.mark.parametrize("precision", ["df32", "fp32", "fp64", "mixed"])
def test_entry_points_agree(oracle, n, precision):
    nb = 3
    plan = Plan(n, LO, HI, precision=precision, max_batch=nb)
    host = [torch.from_numpy(r).to(plan.dtype) for r in _rhs(n, nb)]
    rho = torch.stack(host).cuda()
    alone = torch.stack([plan.solve(rho[b].contiguous()) for b in range(nb)])
    # batched
    assert torch.equal(plan.solve_batched(rho), alone)
    # captured graph, replayed on its own stream after the solves above
    out = torch.full_like(rho, float("nan"))
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        graph = plan.capture(rho, out, stream)
        graph.launch(stream)
    stream.synchronize()
    graph.close()
    assert torch.equal(out, alone)
    # host-resident inputs and outputs through sp_solve_host
    ins = [h.pin_memory() for h in host]
    outs = [torch.empty(n, dtype=plan.dtype).pin_memory() for _ in range(nb)]
    plan.solve_host_stream(ins, outs)
    for b in range(nb):
        assert torch.equal(outs[b], alone[b].cpu())
    plan.sync()
    plan.close()
    # one right-hand side against the oracle
    _, _, M = oracle.plan_tables(n, LO, HI)
    ref = oracle.solve(M, host[1].double().numpy())
    got = alone[1].double().cpu().numpy()
    assert np.abs(got - ref).max() / np.abs(ref).max() <= TOL[precision]
