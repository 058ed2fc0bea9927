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
    # a multiplicity of 0 or above 256 and a radial MLP width of 48 are invalid
    c, _keep = make_config(dataclasses.replace(MODEL_TINY, mul=(0, 32)))
    assert lib.sevennet_n_params(ctypes.byref(c)) < 0
    c, _keep = make_config(dataclasses.replace(MODEL_TINY, mul=(32, 288)))
    assert lib.sevennet_n_params(ctypes.byref(c)) < 0
    with pytest.raises(sn.SevenNetError):
        sn.n_params(dataclasses.replace(MODEL_TINY, mlp_hidden=48))


def _small_specs():
    import dataclasses
    from synth import benchmark_model
    return (benchmark_model(3, 8, lmax=3), benchmark_model(2, 4), benchmark_model(5, 16, lmax=3),
            dataclasses.replace(MODEL_SEVENNET0, mul=(48, 16, 8)))


def test_small_multiplicities_count_like_the_oracle(lib):
    # any multiplicity in [1, 256] is accepted and counted in the canonical (unpadded) layout
    import paper_2402_03789_gb300 as sn
    for spec in _small_specs():
        assert sn.n_params(spec) == oracle.n_params(spec)


def test_library_padding_is_exact_in_the_oracle(lib):
    # the library runs a model with multiplicities that are not multiples of 32
    # as the zero-padded model of sevennet_padded_weights; in the FP64 oracle the
    # padded model has the same E, F and W (the added channels stay zero) and the
    # padded vector has the padded configuration's parameter count
    import dataclasses
    from synth import benchmark_model, make_quartz, normal_weights
    from paper_2402_03789_gb300.model import padded_model
    s = make_quartz("quartz_216")
    for spec in (benchmark_model(2, 8, lmax=2), benchmark_model(2, 4, lmax=3),
                 dataclasses.replace(MODEL_TINY, mul=(20, 12))):
        w = normal_weights(oracle.n_params(spec))
        mul_p, w_p = padded_model(spec, w)
        assert all(m % 32 == 0 for m in mul_p) and len(mul_p) == len(spec.mul)
        spec_p = dataclasses.replace(spec, mul=mul_p)
        assert w_p.size == oracle.n_params(spec_p)
        E, F, W, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
        Ep, Fp, Wp, *_ = oracle.energy_forces_virial(spec_p, w_p, s.species, s.pos, s.cell)
        assert abs(Ep - E) <= 1e-9 * max(1.0, abs(E))
        assert np.abs(Fp - F).max() <= 1e-9 * max(1e-12, np.abs(F).max())
        assert np.abs(Wp - W).max() <= 1e-9 * max(1e-12, np.abs(W).max())
