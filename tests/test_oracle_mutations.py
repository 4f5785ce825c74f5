"""The oracle's pins catch plausible mistakes.  Each case copies the oracle into a
temporary directory, plants one mistake in its C source (a dropped term, a wrong scale,
a flipped sign, a wrong constant), builds that copy, and checks that one of the pins of
tests/test_oracle_*.py fails on it.  Nothing here touches the real oracle or a GPU."""
import importlib.util
import os
import shutil

import pytest

from tests import test_oracle_fft as T_fft
from tests import test_oracle_multiplier as T_mult
from tests import test_oracle_quadrature as T_quad
from tests import test_oracle_solve as T_solve

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _asymptote(o):
    T_mult.test_multiplier_asymptote(o, (24, 32, 20), (-1, -2, -0.5), (1.5, 1, 1))


def _fft(o):
    T_fft.test_fft_vs_brute_force_and_numpy(o, 12, -1)


def _gs(o):
    T_quad.test_gs_table_closed_form_entries(o)
    T_quad.test_gs_ratio_long_double_matches_mpmath(o)


def _table1(o):
    T_solve.test_unit_box_gaussian_scale_invariance(o)


MUTATIONS = [
    ("dropped rank-3 term of the GS transform",
     "v += w[s] * (h0 * g1 * g2 + g0 * h1 * g2 + g0 * g1 * h2);",
     "v += w[s] * (h0 * g1 * g2 + g0 * h1 * g2);", _asymptote),
    ("wavenumber scale off by two on one axis",
     "double kap0 = OR_PI * k0 / L[0];", "double kap0 = 2.0 * OR_PI * k0 / L[0];", _asymptote),
    ("sign of the Laplacian symbol",
     "-(kap0 * kap0 + kap1 * kap1 + kap2 * kap2) * v;", "(kap0 * kap0 + kap1 * kap1 + kap2 * kap2) * v;",
     _table1),
    ("conjugated twiddles", "tw[2 * q + 1] = sign * sin(ang);", "tw[2 * q + 1] = -sign * sin(ang);", _fft),
    ("GS weight missing its 2/sqrt(pi)",
     "w[s] = (1.0 / (8.0 * OR_PI)) * (2.0 / sqrt(OR_PI)) * h_tau * exp(tau);",
     "w[s] = (1.0 / (8.0 * OR_PI)) * h_tau * exp(tau);", _gs),
]


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new, pin):
    d = tmp_path / "oracle_mutant"
    d.mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "__init__.py")
    src = open(os.path.join(ROOT, "oracle", "sp_oracle.c")).read()
    assert src.count(old) == 1, "the mutation site moved"
    (d / "sp_oracle.c").write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{abs(hash(name))}", d / "__init__.py",
                                                  submodule_search_locations=[str(d)])
    mutant = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mutant)
    mutant.build()
    with pytest.raises(AssertionError):
        pin(mutant)
