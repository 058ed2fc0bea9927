"""Host-side checks of the C ABI: the library loads without a GPU, exports
every entry point declared in include/sevennet.h, and its host-only planning
(weight layout) agrees with the oracle's parameter count."""

import os
import re

import pytest

import oracle
from synth import MODEL_SEVENNET0, MODEL_SEVENNET0_89, MODEL_TINY

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sevennet.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sevennet_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_03789_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2402_03789_gb300.build import build
        build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_2402_03789_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(names)


@pytest.mark.parametrize("spec", [MODEL_TINY, MODEL_SEVENNET0, MODEL_SEVENNET0_89])
def test_library_weight_layout_matches_oracle(lib, spec):
    import paper_2402_03789_gb300 as sn
    assert sn.n_params(spec) == oracle.n_params(spec)


def test_invalid_config_rejected(lib):
    import dataclasses
    import paper_2402_03789_gb300 as sn
    bad = dataclasses.replace(MODEL_TINY, mul=(30, 32))
    with pytest.raises(sn.SevenNetError):
        sn.n_params(bad)
