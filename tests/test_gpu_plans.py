"""Every compiled radix plan of the register-resident passes against the FP64 oracle.

The passes pick a radix plan per arithmetic type, padded length 2n and pass kind (z
passes, y line passes, the x pass with the multiplier), and at some lengths a persistent
cp.async-pipelined line kernel.  Each case here puts one padded length on one axis and
keeps the other two at 2n = 64, so that the oracle (Alg. 2 on the full padded grid)
stays cheap while the case still spans many CTAs and ragged column tiles (n2 + 1 = 33
columns).  Each case runs in every precision, first with the built-in tiles (which
select the pipelined kernel where it fits) and then with the autotuned ones, and is
compared with the oracle element by element: FP64 and double-float to 1e-12, FP32 and
mixed to 1e-5, max-norm relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan  # noqa: E402

TOL = {"fp64": 1e-12, "df32": 1e-12, "fp32": 1e-5, "mixed": 1e-5}
LENGTHS = (64, 128, 192, 256, 384, 512, 1024)
LO, HI = (-1.0, -1.1, -0.9), (1.0, 1.2, 0.8)


def _cases():
    out = []
    for axis in range(3):
        for N in LENGTHS:
            n = [32, 32, 32]
            n[axis] = N // 2
            if axis > 0 and N == 64:
                continue  # (32, 32, 32) is the axis-0 case
            out.append(tuple(n))
    return out


_oracle = {}  # every case's density and oracle potential (a few MB each), kept for all precisions


def _reference(oracle, n):
    if n not in _oracle:
        rng = np.random.default_rng(sum(n) + 17 * n[0])
        rho = rng.standard_normal(n)  # white noise: every wavenumber, every register slot
        _, _, M = oracle.plan_tables(n, LO, HI)
        _oracle[n] = (rho, oracle.solve(M, rho))
    return _oracle[n]


@pytest.mark.parametrize("n", _cases())
@pytest.mark.parametrize("precision", ["fp64", "df32", "fp32", "mixed"])
def test_radix_plan_matches_oracle(oracle, n, precision):
    rho, ref = _reference(oracle, n)
    plan = Plan(n, LO, HI, precision=precision)
    t = torch.from_numpy(rho).to("cuda", dtype=plan.dtype)
    scale = np.abs(ref).max()
    u_default = plan.solve(t).double().cpu().numpy()
    assert np.abs(u_default - ref).max() / scale <= TOL[precision], "built-in tiles"
    cfg = plan.autotune(1)
    u_tuned = plan.solve(t).double().cpu().numpy()
    assert np.abs(u_tuned - ref).max() / scale <= TOL[precision], ("autotuned", cfg)
    if cfg["line_plan"] == (0, 0, 0):
        # tiles regroup lines into CTAs and never change a line's arithmetic
        assert np.array_equal(u_default, u_tuned), cfg
    plan.sync()
    plan.close()


# FP32 and mixed at 2n = 256, 512, 1024 and double-float at 256 have an alternative radix
# plan for the line passes (x pass, y passes), which the autotuner may choose.
ALT = {"fp32": (256, 512, 1024), "mixed": (256, 512, 1024), "df32": (256,)}


def _alt_cases():
    out = []
    for precision, lengths in ALT.items():
        for N in lengths:
            for axis in (0, 1):
                n = [32, 32, 32]
                n[axis] = N // 2
                out.append((precision, tuple(n), axis))
    return out


@pytest.mark.parametrize("precision,n,axis", _alt_cases())
def test_alternative_radix_plan_matches_oracle(oracle, precision, n, axis):
    rho, ref = _reference(oracle, n)
    plan = Plan(n, LO, HI, precision=precision)
    line_plan = [0, 0, 0]
    line_plan[axis] = 1
    for tile in (0, 2):  # built-in tile (the pipelined kernel where it fits) and a runtime tile
        line = [0, 0, 0]
        line[axis] = tile
        plan.set_launch_config(line=line, line_plan=line_plan)
        cfg = plan.launch_config()
        assert cfg["line_plan"][axis] == 1
        u = plan.solve(torch.from_numpy(rho).to("cuda", dtype=plan.dtype)).double().cpu().numpy()
        assert np.abs(u - ref).max() / np.abs(ref).max() <= TOL[precision], cfg
    plan.sync()
    plan.close()


def test_launch_config_rejects_absent_plans():
    from paper_2506_04489_gb300._native import SuperpotError
    plan = Plan((64, 32, 32), LO, HI, precision="fp64")  # no alternative plans in native FP64
    with pytest.raises(SuperpotError) as e:
        plan.set_launch_config(line_plan=(1, 0, 0))
    assert e.value.status == "SP_ERR_UNSUPPORTED_SIZE"
    plan.close()
