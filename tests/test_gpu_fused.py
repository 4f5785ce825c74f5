"""The three-pass FP32 schedule: fused plane passes (the z and y transforms of an x-plane
in one launch of 8-CTA clusters exchanging through distributed shared memory), the x
pass, and the fused inverse plane pass.  Checked against the oracle on a grid whose y and z
lengths take the fused passes (2n1 = 2n2 = 512) with another x length, batched against
alone, and refused where it does not exist.  The full-size cases at 256^3 are in
test_gpu_oracle_fullsize.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan, workloads as W  # noqa: E402
from paper_2506_04489_gb300._native import SuperpotError  # noqa: E402

LO, HI = (-1.0, -1.2, -0.9), (1.0, 1.1, 0.8)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_fused_planes_match_oracle(oracle, precision):
    n = (96, 256, 256)  # x length 192 (radix 3), y and z 512
    rng = np.random.default_rng(11)
    rho = W.gaussian_mixture(n, LO, HI, 4) + 0.05 * rng.standard_normal(n)
    _, _, M = oracle.plan_tables(n, LO, HI)
    ref = oracle.solve(M, rho)
    plan = Plan(n, LO, HI, precision=precision)
    plan.set_launch_config(schedule="fused_planes")
    assert plan.launch_config()["schedule"] == "fused_planes"
    u = plan.solve(torch.from_numpy(rho).to("cuda", dtype=plan.dtype)).double().cpu().numpy()
    plan.sync()
    plan.close()
    assert np.abs(u - ref).max() / np.abs(ref).max() <= 1e-5


def test_fused_batched_equals_alone():
    n, nb = (32, 256, 256), 3
    plan = Plan(n, -1.0, 1.0, precision="fp32", max_batch=nb)
    plan.set_launch_config(schedule="fused_planes")
    rhos = torch.stack([torch.from_numpy(W.gaussian_mixture(n, -1.0, 1.0, s)) for s in range(nb)]).float().cuda()
    ub = plan.solve_batched(rhos)
    for b in range(nb):
        assert torch.equal(plan.solve(rhos[b].contiguous()), ub[b])
    plan.sync()
    plan.close()


def test_fused_refused_where_absent():
    for n, precision in (((64, 64, 64), "fp32"), ((32, 256, 256), "df32"), ((32, 256, 128), "fp32")):
        plan = Plan(n, -1.0, 1.0, precision=precision)
        with pytest.raises(SuperpotError) as e:
            plan.set_launch_config(schedule="fused_planes")
        assert e.value.status == "SP_ERR_UNSUPPORTED_SIZE", (n, precision)
        plan.close()
