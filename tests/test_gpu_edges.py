"""Edge cases of the grid, in every precision.

The smallest grids (n = 2) and a moderate Bluestein length (2n = 254) against the oracle
(FP64 and double-float 1e-12, FP32 and mixed 1e-5, max-norm relative).  The largest
padded lengths (2n = 2048 on radix stages; 2n = 2042, twice a prime, on Bluestein's
algorithm with the largest convolution, M = 4096) on the x, y and z axes, where the
oracle's quadrature of the 1D tables is too slow, through a property that holds exactly
at any size: the padded solve is the aperiodic discrete convolution of the density with
the kernel table, so a density shifted by one cell along an axis (its last slab zero
before the shift) has the potential shifted by one cell.  The two solves compared are each
held to the parity tolerance, so their difference is bounded by twice it; the density is
positive (uniform in [0, 1)), so that the potential is not small beside the sums that
form it.  And a zero density gives a zero potential.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2506_04489_gb300 import Plan  # noqa: E402

TOL = {"fp64": 1e-12, "df32": 1e-12, "fp32": 1e-5, "mixed": 1e-5}
PRECISIONS = ["fp64", "df32", "fp32", "mixed"]
LO, HI = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
_ref = {}


def _solve(n, precision, rho):
    plan = Plan(n, LO, HI, precision=precision)
    u = plan.solve(torch.from_numpy(rho).to("cuda", dtype=plan.dtype)).double().cpu().numpy()
    plan.sync()
    plan.close()
    return u


@pytest.mark.parametrize("n", [(2, 2, 2), (2, 3, 5), (3, 2, 2), (8, 127, 8)])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_small_grids_match_oracle(oracle, n, precision):
    if n not in _ref:
        rho = np.random.default_rng(sum(n)).standard_normal(n)
        _, _, M = oracle.plan_tables(n, LO, HI)
        _ref[n] = (rho, oracle.solve(M, rho))
    rho, ref = _ref[n]
    u = _solve(n, precision, rho)
    assert np.abs(u - ref).max() / np.abs(ref).max() <= TOL[precision]


@pytest.mark.parametrize("n,axis", [((1024, 8, 8), 0), ((8, 1024, 8), 1), ((8, 8, 1024), 2),
                                    ((1021, 8, 8), 0), ((8, 8, 1021), 2)])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_largest_lengths_shift_by_one_cell(n, axis, precision):
    rho = np.random.default_rng(sum(n) + axis).random(n)
    last = [slice(None)] * 3
    last[axis] = -1
    rho[tuple(last)] = 0.0
    shifted = np.roll(rho, 1, axis=axis)  # the zero slab wraps to the front
    u = _solve(n, precision, rho)
    us = _solve(n, precision, shifted)
    head, tail = [slice(None)] * 3, [slice(None)] * 3
    head[axis], tail[axis] = slice(1, None), slice(None, -1)
    assert np.abs(us[tuple(head)] - u[tuple(tail)]).max() / np.abs(u).max() <= 2 * TOL[precision]


@pytest.mark.parametrize("n", [(32, 32, 32), (11, 13, 17)])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_zero_density_gives_zero(n, precision):
    plan = Plan(n, -1.0, 1.0, precision=precision)
    u = plan.solve(torch.zeros(n, dtype=plan.dtype, device="cuda"))
    plan.sync()
    plan.close()
    assert torch.count_nonzero(u).item() == 0
