"""Host-side checks of the C ABI: the library loads without a GPU, exports
every entry point declared in include/sevennet.h, and its host-only planning
(weight layout) agrees with the oracle's parameter count."""

import os
import re

import numpy as np
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
    import ctypes
    import paper_2402_03789_gb300 as sn
    from paper_2402_03789_gb300.model import make_config
    # the C ABI takes multiplicities that are multiples of 32 only (the Python
    # binding pads smaller ones, exactly); a radial MLP width of 48 is invalid
    c, _keep = make_config(dataclasses.replace(MODEL_TINY, mul=(30, 32)))
    assert lib.sevennet_n_params(ctypes.byref(c)) < 0
    with pytest.raises(sn.SevenNetError):
        sn.n_params(dataclasses.replace(MODEL_TINY, mlp_hidden=48))


def test_padding_walker_matches_oracle_layout():
    # models with fewer than 32 channels run zero-padded: the binding's walk of
    # the canonical weight layout must count exactly the oracle's parameters
    import dataclasses
    import oracle
    from synth import MODEL_SEVENNET0, benchmark_model
    from paper_2402_03789_gb300 import padding
    for spec in (benchmark_model(3, 8, lmax=3), benchmark_model(2, 4), benchmark_model(5, 16, lmax=3),
                 dataclasses.replace(MODEL_SEVENNET0, mul=(48, 16, 8))):
        assert padding.n_params(spec) == oracle.n_params(spec)
        spec_p, w_p = padding.pad_model(spec, np.arange(oracle.n_params(spec), dtype=np.float64))
        assert all(m % 32 == 0 for m in spec_p.mul)
        assert w_p.size == oracle.n_params(spec_p)


def test_padded_model_is_exact_in_the_oracle():
    # zero-padding a small-channel model to multiples of 32 leaves E, F and W
    # unchanged: the padded channels stay zero through every operation
    from synth import benchmark_model, make_quartz, normal_weights
    from paper_2402_03789_gb300 import padding
    s = make_quartz("quartz_216")
    for spec in (benchmark_model(2, 8, lmax=2), benchmark_model(2, 4, lmax=3)):
        w = normal_weights(oracle.n_params(spec))
        spec_p, w_p = padding.pad_model(spec, w)
        E, F, W, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
        Ep, Fp, Wp, *_ = oracle.energy_forces_virial(spec_p, w_p, s.species, s.pos, s.cell)
        assert abs(Ep - E) <= 1e-9 * max(1.0, abs(E))
        assert np.abs(Fp - F).max() <= 1e-9 * max(1e-12, np.abs(F).max())
        assert np.abs(Wp - W).max() <= 1e-9 * max(1e-12, np.abs(W).max())
