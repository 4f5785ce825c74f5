"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (max-norm relative, as eq. error_infty but against the oracle):
FP64 1e-12, FP32 and mixed 1e-5.  Setup tables (Alg. 1, all FP64 on the GPU) are
compared entry by entry: GS table to 4e-14 relative (exp of a node rounded once), 1D
integrals to 1e-13 of each row's kappa = 0 value, the multiplier to 1e-13 of its maximum.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan, workloads as W  # noqa: E402

TOL = {"fp64": 1e-12, "df32": 1e-12, "fp32": 1e-5, "mixed": 1e-5}


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


_oracle_cache = {}


def oracle_tables(oracle, n, lo, hi):
    key = (tuple(n), tuple(lo), tuple(hi))
    if key not in _oracle_cache:
        _oracle_cache[key] = oracle.plan_tables(n, lo, hi)
    return _oracle_cache[key]


def gpu_solve(n, lo, hi, rho, precision):
    plan = Plan(n, lo, hi, precision=precision)
    t = torch.from_numpy(rho).to("cuda", dtype=plan.dtype)
    u = plan.solve(t)
    torch.cuda.synchronize()
    out = u.double().cpu().numpy()
    plan.close()
    return out


def random_density(n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(n)


CASES = [
    ((8, 8, 8), (-1, -1, -1), (1, 1, 1)),
    ((12, 12, 12), (-1, -1, -1), (1, 1, 1)),       # 2n = 24 = 8 x 3
    ((16, 24, 18), (-1, -2, -1.5), (1, 1, 2.5)),   # anisotropic grid and box, 2n = 36
    ((32, 32, 32), (-1, -1, -1), (1, 1, 1)),       # unit-box Gaussian geometry
    ((48, 48, 48), (-1, -1, -1), (1, 1, 1)),       # 2n = 96 = 8 x 4 x 3
    ((64, 48, 36), (-2, -2, -2), (2, 2, 2)),
    ((96, 96, 96), (-1, -1, -1), (1, 1, 1)),       # 2n = 192 = 8 x 8 x 3
    ((128, 128, 128), (-1, -1, -1), (1, 1, 1)),    # 128^3 workload
    ((10, 14, 20), (-1, -1, -1), (1, 1, 1)),       # 2n = 20, 28, 40: radix-5 and radix-7 stages
    ((35, 25, 40), (-1, -1, -1.5), (1, 1.5, 1)),   # 2n = 70 = 2 x 5 x 7, 50 = 2 x 5 x 5, 80
    ((80, 80, 80), (-1, -1, -1), (1, 1, 1)),       # 2n = 160 = 8 x 4 x 5
    ((112, 70, 98), (-1, -1, -1), (1, 1, 1)),      # 2n = 224 = 8 x 4 x 7, 140, 196 = 4 x 7 x 7
    ((11, 13, 17), (-1, -1, -1), (1, 1, 1)),       # 2n = 22, 26, 34: Bluestein on every axis
    ((22, 16, 61), (-1, -1.5, -1), (1, 1, 2)),     # 2n = 44 = 4 x 11, 32 (radix), 122 = 2 x 61 (Bluestein)
]


@pytest.mark.parametrize("n,lo,hi", CASES)
def test_setup_tables_match_oracle(oracle, n, lo, hi):
    plan = Plan(n, lo, hi, precision="fp64")
    w, a, M = oracle_tables(oracle, n, lo, hi)
    _, L = oracle.geometry(n, lo, hi)
    for axis in range(3):
        t = plan.tables(axis)
        assert len(t["gs_w"]) == len(w)
        # tau_s = tau_lo + s h may round differently (fused multiply-add on the GPU);
        # exp turns an absolute tau error of |tau| 2^-52 (|tau| < 45) into that relative error
        np.testing.assert_allclose(t["gs_w"], w, rtol=2e-14, atol=0)
        np.testing.assert_allclose(t["gs_a"], a, rtol=4e-14, atol=0)
        G, H = oracle.axis_tables(n[axis], L[axis], a)
        sg = np.abs(G[:, :1])
        sh = np.abs(H[:, :1])
        assert np.all(np.abs(t["G"] - G) <= 1e-13 * sg + 1e-300)
        assert np.all(np.abs(t["H"] - H) <= 1e-13 * sh + 1e-300)
    Ntil = 8.0 * n[0] * n[1] * n[2]
    assert np.abs(t["M"] - M / Ntil).max() <= 1e-13 * np.abs(M / Ntil).max()
    assert t["M"][0, 0, 0] == 0.0
    plan.close()


def mixture_density(n, lo, hi, seed):
    """Seeded Gaussian mixture on the case's box, centres scaled into the box."""
    centres, sig, wts = W.mixture_params(seed)
    c = np.asarray(lo, float) / 2 + np.asarray(hi, float) / 2
    half = (np.asarray(hi, float) - np.asarray(lo, float)) / 2
    out = np.zeros(n)
    for cc, s, w_ in zip(centres, sig, wts):
        out += w_ * W.gaussian(n, lo, hi, s * float(half.min()), c + cc * half)
    return out


@pytest.mark.parametrize("n,lo,hi", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed", "df32"])
def test_solve_matches_oracle(oracle, n, lo, hi, precision):
    # double-float runs the register-resident passes where every padded length has a
    # compiled plan and the first-generation passes (radix 2 to 8, 3, 5, 7) elsewhere
    rho = mixture_density(n, lo, hi, sum(n))
    _, _, M = oracle_tables(oracle, n, lo, hi)
    ref = oracle.solve(M, rho)
    u = gpu_solve(n, lo, hi, rho, precision)
    assert _rel(u, ref) <= TOL[precision]


@pytest.mark.parametrize("n,lo,hi", CASES)
def test_white_noise_matches_oracle(oracle, n, lo, hi):
    # White noise weights every wavenumber equally, so it exercises the multiplier at
    # high |k|, where G and H are far below the size of their integrands (both sides
    # take them in the integrated-by-parts form there).
    rho = random_density(n, sum(n))
    _, _, M = oracle_tables(oracle, n, lo, hi)
    ref = oracle.solve(M, rho)
    u = gpu_solve(n, lo, hi, rho, "fp64")
    assert _rel(u, ref) <= 1e-12
    u32 = gpu_solve(n, lo, hi, rho, "fp32")
    assert _rel(u32, ref) <= 1e-5
    udf = gpu_solve(n, lo, hi, rho, "df32")
    assert _rel(udf, ref) <= 1e-12


def test_unit_box_gaussian_fp64_and_analytic(oracle):
    from tests import analytic as A
    n, lo, hi = 32, -1.0, 1.0
    rho = W.gaussian(n, lo, hi, 0.1)
    _, _, M = oracle_tables(oracle, (n,) * 3, (lo,) * 3, (hi,) * 3)
    ref = oracle.solve(M, rho)
    u = gpu_solve((n,) * 3, (lo,) * 3, (hi,) * 3, rho, "fp64")
    assert _rel(u, ref) <= 1e-12
    E = A.rel_err(u, A.gaussian_u(n, lo, hi, 0.1))
    assert abs(E / 4.154e-9 - 1) < 0.02  # Tab. 1, sigma = 0.2, n = 32 row, scaled box


@pytest.mark.parametrize("dens", ["cos_gaussian", "bump"])
def test_128_workload_densities(oracle, dens):
    n, lo, hi = (128,) * 3, (-1.0,) * 3, (1.0,) * 3
    rho = W.cos_gaussian(128, -1.0, 1.0) if dens == "cos_gaussian" else W.bump_profile(128, -1.0, 1.0)
    _, _, M = oracle_tables(oracle, n, lo, hi)
    ref = oracle.solve(M, rho)
    for precision in ("fp64", "fp32"):
        u = gpu_solve(n, lo, hi, rho, precision)
        assert _rel(u, ref) <= TOL[precision], precision


@pytest.mark.parametrize("n", [(16, 24, 18), (32, 64, 32), (96, 32, 64), (13, 8, 11)])
@pytest.mark.parametrize("precision", ["fp64", "df32", "fp32"])
def test_forward_spectrum_matches_oracle(oracle, n, precision):
    lo, hi = (-1, -1, -1), (1, 1, 1)
    rho = random_density(n, 7)
    plan = Plan(n, lo, hi, precision=precision)
    spec = plan.forward_spectrum(torch.from_numpy(rho).cuda().to(plan.dtype))
    torch.cuda.synchronize()
    got = spec.cpu().numpy()
    if precision == "df32":  # four float32 per value: re.hi, im.hi, re.lo, im.lo
        got = got.astype(np.float64)
        got = (got[..., 0] + got[..., 2]) + 1j * (got[..., 1] + got[..., 3])
    ref = oracle.forward_spectrum(rho)
    # FP32 passes on FP32 input: the input rounding alone is 2^-24 of each value
    tol = 1e-6 if precision == "fp32" else 1e-13
    assert np.abs(got - ref).max() <= tol * np.abs(rho).sum()
    plan.close()


def test_batched_equals_single(oracle):
    n, lo, hi = (32, 32, 32), (-1,) * 3, (1,) * 3
    plan = Plan(n, lo, hi, precision="fp64", max_batch=4)
    rhos = torch.stack([torch.from_numpy(W.gaussian_mixture(32, -1, 1, s)) for s in range(4)]).cuda()
    ub = plan.solve_batched(rhos)
    for b in range(4):
        us = plan.solve(rhos[b].contiguous())
        assert torch.equal(us, ub[b])
    plan.close()


def test_in_place_alias(oracle):
    n, lo, hi = (24, 24, 24), (-1,) * 3, (1,) * 3
    rho = random_density(n, 3)
    plan = Plan(n, lo, hi, precision="fp64")
    t = torch.from_numpy(rho).cuda()
    ref = plan.solve(t.clone())
    plan.solve(t, out=t)
    assert torch.equal(t, ref)
    plan.close()


def test_explicit_gs_table_matches_generated(oracle):
    n, lo, hi = (18, 18, 18), (-1,) * 3, (1,) * 3
    _, L = oracle.geometry(n, lo, hi)
    w, a = oracle.gs_table(1e-4, oracle.default_delta(L))
    rho = random_density(n, 11)
    p1 = Plan(n, lo, hi, precision="fp64")
    p2 = Plan(n, lo, hi, precision="fp64", gs=(w, a))
    t = torch.from_numpy(rho).cuda()
    u1, u2 = p1.solve(t), p2.solve(t)
    assert float((u1 - u2).abs().max() / u1.abs().max()) <= 1e-14
    p1.close()
    p2.close()


def test_not_ready_and_batch_errors():
    from paper_2506_04489_gb300._native import SuperpotError
    plan = Plan(8, -1, 1, precision="fp64", precompute=False, max_batch=2)
    t = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(SuperpotError) as e:
        plan.solve(t)
    assert e.value.status == "SP_ERR_NOT_READY"
    plan.precompute()
    with pytest.raises(SuperpotError) as e:
        plan.solve_batched(torch.zeros((3, 8, 8, 8), dtype=torch.float64, device="cuda"))
    assert e.value.status == "SP_ERR_INVALID"
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "df32", "fp32"])
def test_plain_gs_kernel_matches_oracle(oracle, precision):
    n, lo, hi = (64, 64, 64), (-2.0,) * 3, (2.0,) * 3
    rho = W.gaussian(64, -2.0, 2.0, 0.2)
    _, _, M = oracle.plan_tables(n, lo, hi, kernel="gs_plain")
    ref = oracle.solve(M, rho)
    plan = Plan(n, lo, hi, precision=precision, kernel="gs_plain")
    u = plan.solve(torch.from_numpy(rho).cuda().to(plan.dtype)).double().cpu().numpy()
    plan.close()
    assert _rel(u, ref) <= TOL[precision]
