"""The shapes of the paper's scaling benchmarks (Sec. 4: r_c 4 A, equal
channels for every irrep, 2-5 layers, lmax 2 and the paper's lmax 3) against
the FP64 oracle on a 216-atom cell at the alpha-quartz density, FP32 and BF16
paths."""

import numpy as np
import pytest

import oracle
from synth import benchmark_model, make_quartz, normal_weights
from gpu_common import errors, get_model

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_layers,channels,lmax", [(2, 64, 2), (5, 32, 2), (3, 32, 2), (2, 32, 3), (3, 64, 3)])
def test_benchmark_shape_matches_oracle(n_layers, channels, lmax):
    s = make_quartz("quartz_216")
    spec = benchmark_model(n_layers, channels, lmax=lmax)
    model = get_model(spec)
    w = normal_weights(oracle.n_params(spec))
    Eo, Fo, Wo, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
    E, F, W = model.evaluate(s.pos, s.cell, s.species, "fp32")
    e_pa, f_rel, w_rel = errors(E, F, W, Eo, Fo, Wo, s.n_atoms)
    assert e_pa <= 1e-6 and f_rel <= 1e-5 and w_rel <= 1e-5, (e_pa, f_rel, w_rel)
    E, F, W = model.evaluate(s.pos, s.cell, s.species, "bf16")
    e_pa, f_rel, w_rel = errors(E, F, W, Eo, Fo, Wo, s.n_atoms)
    print(f"bf16 {n_layers}x{channels} lmax {lmax}: |dE|/N={e_pa:.2e} F={f_rel:.2e} W={w_rel:.2e}")
    # energy and virial bounds from the measured errors of these shapes (at most
    # 6.1e-6 eV/atom and 3.4e-3) with a margin of about 3x
    assert f_rel <= 5e-3 and e_pa <= 2e-5 and w_rel <= 1e-2, (e_pa, f_rel, w_rel)


@pytest.mark.parametrize("n_layers,channels,lmax", [(2, 4, 3), (3, 8, 3), (3, 16, 2)])
def test_small_channel_models_match_oracle(n_layers, channels, lmax):
    # the paper's 4-16 channel models, created through the C ABI from their own
    # (unpadded) weights; the library runs them as the exact zero-padded model
    s = make_quartz("quartz_216")
    spec = benchmark_model(n_layers, channels, lmax=lmax)
    import paper_2402_03789_gb300 as sn
    w = normal_weights(oracle.n_params(spec))
    model = sn.SevenNet(spec, w)
    Eo, Fo, Wo, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
    E, F, W = model.evaluate(s.pos, s.cell, s.species, "fp32")
    e_pa, f_rel, w_rel = errors(E, F, W, Eo, Fo, Wo, s.n_atoms)
    assert e_pa <= 1e-6 and f_rel <= 1e-5 and w_rel <= 1e-5, (e_pa, f_rel, w_rel)
    model.close()
