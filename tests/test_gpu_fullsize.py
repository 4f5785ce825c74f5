"""Parity at the full workload sizes (256^3 and 512^3 on [-1,1]^3), where the oracle
cannot run the whole solve:

* the forward padded spectrum (first step of Alg. 2) at sampled wavenumbers against the
  oracle's direct summation, one coefficient at a time;
* the potential of the C-infinity bump density against its radial-quadrature solution
  (Newton's shell theorem) at sampled grid points;
* translation: shifting the density by one grid cell shifts the potential by one cell;
* double-float and mixed precision against the native FP64 path on the same input.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan, workloads as W  # noqa: E402
from tests import analytic as A  # noqa: E402

LO, HI, R = -1.0, 1.0, 0.8


def _bump(n):
    return torch.from_numpy(W.bump_profile(n, LO, HI, R))


@pytest.mark.parametrize("n", [256, 512])
@pytest.mark.parametrize("precision", ["fp64", "df32"])
def test_sampled_spectrum_coefficients(oracle, n, precision):
    rho = _bump(n).numpy()
    rng = np.random.default_rng(n)
    noise = rng.standard_normal((n, n, n)) * 1e-3  # break the bump's symmetry
    rho = rho + noise * (rho > 0)
    plan = Plan(n, LO, HI, precision=precision)
    spec = plan.forward_spectrum(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    scale = float(np.abs(rho).sum())
    ks = [(0, 0, 0), (n, n, n), (2 * n - 1, 1, n), (1, 2 * n - 1, 0)]
    ks += [tuple(int(v) for v in (rng.integers(2 * n), rng.integers(2 * n), rng.integers(n + 1))) for _ in range(3)]
    for k in ks:
        ref = oracle.dft_coeff(rho, k)
        s = spec[k]
        if precision == "df32":  # (re.hi, im.hi, re.lo, im.lo)
            s = s.double().cpu().numpy()
            got = complex(s[0] + s[2], s[1] + s[3])
        else:
            got = complex(s.item())
        assert abs(got - ref) <= 1e-13 * scale, (k, got, ref)
    plan.close()
    del spec
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [256, 512])
def test_bump_potential_radial_quadrature(n):
    rho = _bump(n).cuda()
    prof = lambda s: math.exp(-1.0 / (1.0 - s * s / (R * R))) if s < R else 0.0
    x = np.linspace(LO, HI, n)
    rng = np.random.default_rng(1)
    idx = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(60)]
    idx += [(n // 2, n // 2, j) for j in range(0, n, max(1, n // 16))]
    ref = np.array([A.radial_potential(prof, R, math.sqrt(sum(x[i] ** 2 for i in p))) for p in idx])
    for precision in ("df32", "fp64"):
        plan = Plan(n, LO, HI, precision=precision)
        u = plan.solve(rho).cpu().numpy()
        got = np.array([u[p] for p in idx])
        E = np.abs(got - ref).max() / np.abs(ref).max()
        # the bump is C-infinity but not analytic: 1.2e-7 at n = 64 on [-1,1]^3, lower above
        assert E < 1e-10, (precision, E)
        plan.close()


def test_translation_shifts_potential():
    n = 256
    rho = _bump(n)
    shifted = torch.zeros_like(rho)
    shifted[1:, :, :] = rho[:-1, :, :]  # one cell along x (the bump is zero near the faces)
    plan = Plan(n, LO, HI, precision="df32")
    u = plan.solve(rho.cuda())
    us = plan.solve(shifted.cuda())
    d = (us[1:] - u[:-1]).abs().max() / u.abs().max()
    assert float(d) <= 1e-12
    plan.close()


@pytest.mark.parametrize("n", [256, 512])
def test_precisions_against_native_fp64(n):
    rho = _bump(n).cuda()
    u = {}
    for precision in ("fp64", "df32", "mixed"):
        plan = Plan(n, LO, HI, precision=precision)
        u[precision] = plan.solve(rho)
        torch.cuda.synchronize()
        plan.close()
    ref = u["fp64"]
    dev = lambda a: float((a - ref).abs().max() / ref.abs().max())
    assert dev(u["df32"]) <= 1e-12
    assert dev(u["mixed"]) <= 1e-5
    for p in ("fp32",):
        plan = Plan(n, LO, HI, precision=p)
        u32 = plan.solve(rho.float()).double()
        plan.close()
        assert dev(u32) <= 1e-5


@pytest.mark.parametrize("n", [128, 256])
def test_spectral_laplacian_returns_the_potential(n):
    # rho = -Laplacian of the C-infinity bump u*, taken spectrally on the padded periodic
    # grid (reference arithmetic with torch.fft in FP64, not the solver): the solve must
    # return u* up to the method's discretisation error (the oracle measures 1.5e-5 at
    # n = 64, falling about as h^4), on every grid point.
    L = n * (HI - LO) / (n - 1)  # window half-width n h
    ustar = _bump(n).cuda()
    m = 2 * n
    P = torch.zeros((m, m, m), dtype=torch.float64, device="cuda")
    P[:n, :n, :n] = ustar
    k = torch.fft.fftfreq(m, 1.0 / m, dtype=torch.float64, device="cuda") * (math.pi / L)
    K2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    rho = torch.fft.ifftn(K2 * torch.fft.fftn(P)).real[:n, :n, :n].contiguous()
    del P, K2
    bound = {128: 2e-6, 256: 2e-7}[n]
    for precision, tol in (("df32", bound), ("fp64", bound), ("fp32", max(bound, 2e-6))):
        plan = Plan(n, LO, HI, precision=precision)
        u = plan.solve(rho.to(plan.dtype)).double()
        E = float((u - ustar).abs().max() / ustar.abs().max())
        assert E < tol, (precision, E)
        plan.close()


@pytest.mark.parametrize("precision", ["df32", "fp32", "fp64"])
def test_benchmark_launch_configuration_bitwise(precision):
    # The benchmark autotunes the tiles (and so runs other kernels: runtime tiles, the
    # pipelined line kernel) before timing; the full-size parity above uses the default
    # tiles.  Tiles only regroup lines into CTAs, so the 256^3 results must agree bit for
    # bit, which carries every full-size check over to the timed configuration.
    n = 256
    plan = Plan(n, LO, HI, precision=precision)
    rho = _bump(n).cuda().to(plan.dtype)
    before = plan.solve(rho)
    cfg = plan.autotune(1)
    after = plan.solve(rho)
    torch.cuda.synchronize()
    if cfg["line_plan"] == (0, 0, 0):
        assert torch.equal(before, after), cfg
    else:  # another radix plan rounds differently: within the precision's bar
        tol = {"df32": 1e-12, "fp32": 1e-5, "fp64": 1e-12}[precision]
        d = float((after.double() - before.double()).abs().max() / before.double().abs().max())
        assert d <= tol, (cfg, d)
    plan.close()
