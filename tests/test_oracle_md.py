"""Pins of the oracle integrator: NVE energy conservation of velocity Verlet
and its second-order error (halving dt quarters the energy error)."""

import dataclasses

import numpy as np

import oracle
from synth import make_workload, normal_weights, maxwell_boltzmann

KB = 8.617333262e-5


def _setup(scale):
    s, spec = make_workload("sio2_192")
    spec = dataclasses.replace(spec, scale=scale)
    w = normal_weights(oracle.n_params(spec))
    m = s.masses()
    v = maxwell_boltzmann(m, 3000.0, seed=3)
    return s, spec, w, m, v


def test_initial_velocities():
    s, spec, w, m, v = _setup(1.0)
    assert abs(oracle.kinetic_energy(v, m) - 0.5 * (3 * len(m) - 3) * KB * 3000) < 1e-9
    assert np.abs((m[:, None] * v).sum(0)).max() < 1e-12


def test_nve_drift_small():
    s, spec, w, m, v = _setup(1.0)
    E0, F0, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
    etot0 = E0 + oracle.kinetic_energy(v, m)
    _, _, _, ep, ek = oracle.velocity_verlet(spec, w, s.species, s.pos, v, m, s.cell, 1.0, 100)
    drift = np.abs(ep + ek - etot0).max() / len(m)
    assert drift < 1e-5, drift


def test_verlet_error_is_second_order():
    # an energy scale of 200 gives O(0.1) eV/A forces, so the error is measurable
    s, spec, w, m, v = _setup(200.0)
    E0, F0, *_ = oracle.energy_forces_virial(spec, w, s.species, s.pos, s.cell)
    assert np.sqrt((F0 ** 2).mean()) > 0.05
    etot0 = E0 + oracle.kinetic_energy(v, m)
    errs = []
    for dt, n in ((1.0, 8), (0.5, 16)):
        _, _, _, ep, ek = oracle.velocity_verlet(spec, w, s.species, s.pos, v, m, s.cell, dt, n)
        errs.append(abs(ep[-1] + ek[-1] - etot0))
    ratio = errs[0] / errs[1]
    assert 2.5 < ratio < 6.0, (errs, ratio)
