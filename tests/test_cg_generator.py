"""The library's build step generates its Clebsch-Gordan tables independently
of the oracle (exact rationals from the Racah formula, its own real-basis map);
every coupling with l <= 3 must equal the oracle's real CG tensor."""

import importlib.util
import os

import numpy as np
import pytest

from oracle.so3 import real_cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _gen():
    spec = importlib.util.spec_from_file_location(
        "gen_cg", os.path.join(ROOT, "paper_2402_03789_gb300", "csrc", "gen_cg.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


COUPLINGS = [(a, b, c) for a in range(4) for b in range(4) for c in range(abs(a - b), min(a + b, 3) + 1)]


@pytest.mark.parametrize("l1,l2,l3", COUPLINGS)
def test_generated_tables_equal_oracle(l1, l2, l3):
    g = _gen()
    tab = g.real_cg_table(l1, l2, l3)
    dense = np.zeros((2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1))
    for (a, b, c), v in tab.items():
        dense[a, b, c] = float(v)
    assert np.abs(dense - real_cg(l1, l2, l3)).max() < 1e-12
